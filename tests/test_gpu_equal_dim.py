"""Equal-dimension variant (Sec. 2.2, Eqs. 10-11) through the C ABI: a
station at the centre of every cell, the three-level Toeplitz product by a
three-level circulant embedding and FFT.

* small odd meshes, every station: grav_forward3d against the CPU oracle's
  direct summation (oracle.forward3d), FP64 <= 1e-10 and FP32 <= 2e-5
  relative L2 per component; grav_adjoint3d against oracle.adjoint3d;
* every transform length of the implementation (x rows up to 2048 points,
  y columns up to 2048, z up to 1024): sampled stations and cells;
* <G x, y> = <x, G^T y>.
"""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan3D

pytestmark = pytest.mark.gpu

ALL7 = 127
TOL64, TOL32 = 1e-10, 2e-5


def _rel(got, ref):
    """Per-component relative L2 error; a component that vanishes by symmetry
    is measured against 1e-3 of the largest norm of the same derivative order
    (as in the plane tests)."""
    g = got.reshape(got.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    num = np.linalg.norm(g - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    return num / np.maximum(den, 1e-3 * den.max())


def _forward(mesh, comps, rho, fp64):
    dt = torch.float64 if fp64 else torch.float32
    with Plan3D(mesh, comps, fp64=fp64) as plan:
        out = plan.forward(torch.as_tensor(rho, dtype=dt).cuda())
        torch.cuda.synchronize()
        return out.cpu().double().numpy()


def _adjoint(mesh, comps, r, fp64):
    dt = torch.float64 if fp64 else torch.float32
    with Plan3D(mesh, comps, fp64=fp64) as plan:
        g = plan.adjoint(torch.as_tensor(r, dtype=dt).cuda())
        torch.cuda.synchronize()
        return g.cpu().double().numpy()


# (5, 4, 70) .. (3, 11, 65) reach the 256-point layer transform (65 <= nz <=
# 128) held in registers, with fewer y columns than one tile of it (ny = 1, 4)
# and a ragged one; (513, 3, 2) the tiled inverse y and x passes of FP32 plans
# with Px = 2048, ny short of one block of 8 rows
SMALL = [(1, 1, 1, 10.0, 10.0, 10.0, 1.0), (5, 4, 3, 20.0, 25.0, 10.0, 1.0), (9, 1, 4, 10.0, 10.0, 15.0, 1.0),
         (3, 11, 2, 12.0, 10.0, 30.0, 1.0), (17, 13, 9, 10.0, 12.0, 8.0, 1.0), (5, 4, 70, 20.0, 25.0, 10.0, 1.0),
         (9, 1, 100, 10.0, 10.0, 15.0, 1.0), (3, 11, 65, 12.0, 10.0, 30.0, 1.0), (513, 3, 2, 10.0, 10.0, 10.0, 1.0)]


@pytest.mark.parametrize("mesh", SMALL)
@pytest.mark.parametrize("fp64,tol", [(True, TOL64), (False, TOL32)])
def test_forward3d_matches_oracle_everywhere(gravlib, orc, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    rho = rng.uniform(-500, 500, (nz, ny, nx))
    if not fp64:
        rho = rho.astype(np.float32).astype(np.float64)
    got = _forward(mesh, ALL7, rho, fp64)
    ref = orc.forward3d(mesh, ALL7, rho)
    err = _rel(got, ref)
    assert np.all(err <= tol), err


@pytest.mark.parametrize("mesh", SMALL[1:])
@pytest.mark.parametrize("fp64,tol", [(True, TOL64), (False, TOL32)])
def test_adjoint3d_matches_oracle_everywhere(gravlib, orc, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx + ny + nz)
    comps = capi.GRAV_ALL6
    r = rng.normal(size=(6, nz, ny, nx))
    if not fp64:
        r = r.astype(np.float32).astype(np.float64)
    got = _adjoint(mesh, comps, r, fp64)
    ref = orc.adjoint3d(mesh, comps, r)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("comps", [capi.GRAV_GZ | capi.GRAV_GX | capi.GRAV_GY, capi.GRAV_GXZ | capi.GRAV_GYZ,
                                   0x1FF & ~capi.GRAV_GZZ])
def test_component_subsets(gravlib, orc, comps):
    """Slot order, the imaginary spectra (gz, gx, gy) and the odd-in-z
    components (gz, gxz, gyz) in every combination."""
    mesh = (7, 6, 5, 10.0, 12.0, 9.0, 1.0)
    rng = np.random.default_rng(comps)
    rho = rng.uniform(-500, 500, (5, 6, 7))
    got = _forward(mesh, comps, rho, True)
    ref = orc.forward3d(mesh, comps, rho)
    assert np.all(_rel(got, ref) <= TOL64)


# every transform length of the implementation: 2048-point x rows (the FP32
# warp-transform row kernel), 2048-point y columns, 1024-point z columns, and
# the register-resident 256-point z columns over many tiles (nz = 128, the
# most that length holds, and nz = 100), the warp-pair 2048-point y transforms
# (513 <= ny <= 1024) and, with 513 <= nx <= 1024 as well, the tiled inverse
# y and x passes
LARGE = [(520, 9, 5, 20.0, 20.0, 10.0, 1.0), (12, 600, 6, 20.0, 15.0, 10.0, 1.0), (6, 5, 300, 20.0, 20.0, 5.0, 1.0),
         (64, 48, 40, 20.0, 20.0, 20.0, 1.0), (40, 36, 128, 20.0, 20.0, 10.0, 1.0), (33, 70, 100, 25.0, 20.0, 10.0, 1.0),
         (600, 13, 70, 20.0, 20.0, 10.0, 1.0), (520, 530, 3, 20.0, 20.0, 10.0, 1.0)]


@pytest.mark.parametrize("mesh", LARGE)
@pytest.mark.parametrize("fp64,tol", [(True, TOL64), (False, TOL32)])
def test_large_sizes_at_sampled_stations(gravlib, orc, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(7)
    m = W.Mesh(*mesh)
    rho = W.serving_density(m, rng, np.float64)
    rho += rng.normal(0, 20, rho.shape)
    if not fp64:
        rho = rho.astype(np.float32).astype(np.float64)
    got = _forward(mesh, capi.GRAV_ALL6, rho, fp64).reshape(6, -1)
    n = nx * ny * nz
    st = np.unique(np.concatenate([[0, n - 1, nx - 1, n - nx, n // 2], rng.choice(n, 11, replace=False)]))
    ref = orc.forward3d(mesh, capi.GRAV_ALL6, rho, stations=st)
    err = _rel(got[:, st], ref)
    assert np.all(err <= tol), err
    # adjoint at sampled cells
    r = rng.normal(size=(6, nz, ny, nx))
    if not fp64:
        r = r.astype(np.float32).astype(np.float64)
    g = _adjoint(mesh, capi.GRAV_ALL6, r, fp64).reshape(-1)
    cells = st[:8]
    gref = orc.adjoint3d(mesh, capi.GRAV_ALL6, r, cells=cells)
    assert np.linalg.norm(g[cells] - gref) <= tol * np.linalg.norm(gref)


@pytest.mark.parametrize("mesh", [(33, 20, 17, 10.0, 10.0, 10.0, 1.0), (20, 18, 90, 10.0, 10.0, 10.0, 1.0),
                                  (530, 10, 6, 10.0, 10.0, 10.0, 1.0), (514, 600, 3, 10.0, 10.0, 10.0, 1.0)])
@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_dot_product_identity(gravlib, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    dt = torch.float64 if fp64 else torch.float32
    gen = torch.Generator().manual_seed(3)
    x = torch.randn((nz, ny, nx), generator=gen, dtype=torch.float64)
    y = torch.randn((6, nz, ny, nx), generator=gen, dtype=torch.float64)
    with Plan3D(mesh, capi.GRAV_ALL6, fp64=fp64) as plan:
        gx = plan.forward(x.to(dt).cuda()).double().cpu()
        gty = plan.adjoint(y.to(dt).cuda()).double().cpu()
    lhs = float((gx * y).sum())
    rhs = float((x * gty).sum())
    assert abs(lhs - rhs) <= tol * np.sqrt(float((gx * gx).sum()) * float((y * y).sum()))


def test_plane_calls_reject_an_equal_dimension_plan(gravlib):
    mesh = (8, 8, 4, 10.0, 10.0, 10.0, 1.0)
    with Plan3D(mesh, capi.GRAV_ALL6) as plan:
        x = torch.zeros((4, 8, 8), device="cuda")
        out = torch.zeros((6, 8, 8), device="cuda")
        assert gravlib.grav_forward(plan.handle, x.data_ptr(), out.data_ptr(), None) == capi.GRAV_EINVAL
        assert "grav_plan_create3d" in capi.grav_last_error()
        info = capi.grav_plan_info(plan.handle)
        assert info.equal_dim == 1 and info.pz == 8
