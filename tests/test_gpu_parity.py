"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Bars (per component, relative L2 over the compared stations or cells):
  FP64 spectral path vs the oracle            <= 1e-10
  FP32 spectral path vs the oracle / FP64     <= 2e-5
Components that vanish by symmetry (e.g. gxz on a one-column mesh) are
compared against a floor of 1e-3 times the largest component norm of the
same kind (first derivatives gz, gx, gy, or the gradients), so rounding
noise in the oracle does not count as a relative error.
"""
import numpy as np
import pytest
import torch

import golden_data
from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan, kernel_values

pytestmark = pytest.mark.gpu

ALL7 = 0x7F
# the six plus the horizontal first derivatives gx, gy (eight components)
ALL7_GXY_SANS_GZZ = 0x3F | capi.GRAV_GX | capi.GRAV_GY
TOL64 = 1e-10
TOL32 = 2e-5


FIRST_DERIV = (0, 7, 8)  # gz, gx, gy (m/s^2); the others are second derivatives (1/s^2)


def rel_errors(got, ref, comps):
    """Relative L2 error per component with a symmetry floor: 1e-3 of the
    largest norm among the components of the same kind (first or second
    derivatives of the potential)."""
    got = np.asarray(got, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    lst = capi.comp_list(comps)
    norms = np.linalg.norm(ref, axis=1)
    kmax = {}
    for i, c in enumerate(lst):
        k = c in FIRST_DERIV
        kmax[k] = max(kmax.get(k, 0.0), norms[i])
    out = []
    for i, c in enumerate(lst):
        floor = 1e-3 * kmax[c in FIRST_DERIV]
        den = max(norms[i], floor, 1e-300)
        out.append(np.linalg.norm(got[i] - ref[i]) / den)
    return np.array(out)


def run_forward(mesh, comps, rho, fp64):
    dt = torch.float64 if fp64 else torch.float32
    with Plan(mesh, comps, fp64=fp64) as plan:
        out = plan.forward(torch.as_tensor(np.asarray(rho), dtype=dt).cuda().contiguous())
        torch.cuda.synchronize()
        return out.cpu().numpy()


def run_adjoint(mesh, comps, r, fp64):
    dt = torch.float64 if fp64 else torch.float32
    with Plan(mesh, comps, fp64=fp64) as plan:
        out = plan.adjoint(torch.as_tensor(np.asarray(r), dtype=dt).cuda().contiguous())
        torch.cuda.synchronize()
        return out.cpu().numpy()


SMALL_MESHES = [
    (16, 16, 4, 10.0, 10.0, 10.0, 1.0),
    (1, 1, 1, 5.0, 5.0, 5.0, 1.0),
    (3, 5, 2, 10.0, 12.0, 8.0, 2.0),
    (17, 9, 3, 25.0, 20.0, 10.0, 3.0),
    (2, 33, 2, 10.0, 10.0, 10.0, 1.0),
    (37, 29, 5, 20.0, 20.0, 15.0, 4.0),
    (64, 1, 3, 10.0, 10.0, 10.0, 2.0),
]


@pytest.mark.parametrize("mesh", [(5, 4, 3, 10.0, 25.0, 20.0, 2.0), (9, 6, 2, 50.0, 50.0, 25.0, 10.0)])
def test_kernel_values_match_oracle(gravlib, orc, mesh):
    """FP64 kernel generation (Eq. 2 and the gradient forms over the offset
    grid of Eq. 10) against the oracle's independent prism evaluation."""
    nx, ny, nz, dx, dy, dz, h = mesh
    for comps in (ALL7, ALL7_GXY_SANS_GZZ):
        lst = capi.comp_list(comps)
        K = kernel_values(mesh, comps).cpu().numpy()
        for n in range(nz):
            for v in range(-ny + 1, ny):
                for u in range(-nx + 1, nx):
                    box = ((u - 0.5) * dx, (u + 0.5) * dx, (v - 0.5) * dy, (v + 0.5) * dy, n * dz, (n + 1) * dz)
                    ref = orc.prism((0.0, 0.0, -h), box)[lst]
                    got = K[:, n, v + ny - 1, u + nx - 1]
                    scale = np.abs(K[:, n]).reshape(len(lst), -1).max(axis=1)
                    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-13 * scale), (n, u, v, got, ref)


@pytest.mark.parametrize("mesh", SMALL_MESHES)
def test_forward_fp64_matches_oracle(gravlib, orc, mesh):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    rho = rng.uniform(-500, 500, (nz, ny, nx))
    got = run_forward(mesh, ALL7, rho, fp64=True)
    ref = orc.forward(mesh, ALL7, rho)
    err = rel_errors(got, ref, ALL7)
    assert np.all(err <= TOL64), err


@pytest.mark.parametrize("mesh", SMALL_MESHES)
def test_forward_fp32_matches_oracle(gravlib, orc, mesh):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz + 1)
    rho = rng.uniform(-500, 500, (nz, ny, nx)).astype(np.float32)
    got = run_forward(mesh, ALL7, rho, fp64=False)
    ref = orc.forward(mesh, ALL7, rho.astype(np.float64))
    err = rel_errors(got, ref, ALL7)
    assert np.all(err <= TOL32), err


@pytest.mark.parametrize("mesh", SMALL_MESHES)
@pytest.mark.parametrize("fp64", [True, False])
def test_adjoint_matches_oracle(gravlib, orc, mesh, fp64):
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx + 7 * ny + 31 * nz)
    r = rng.normal(size=(7, ny, nx))
    if not fp64:
        r = r.astype(np.float32)
    got = run_adjoint(mesh, ALL7, r, fp64)
    ref = orc.adjoint(mesh, ALL7, np.asarray(r, np.float64))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= (TOL64 if fp64 else TOL32), err


@pytest.mark.parametrize("comps", [capi.GRAV_GZ, capi.GRAV_GXZ, capi.GRAV_GYZ, capi.GRAV_GXY,
                                   capi.GRAV_GZ | capi.GRAV_GZZ, capi.GRAV_ALL6, 0b1011010])
def test_component_subsets(gravlib, orc, comps):
    """Any component mask: output planes come in ascending bit order."""
    mesh, rho = W.small16()
    ref = orc.forward(mesh.tuple(), comps, rho)
    got = run_forward(mesh.tuple(), comps, rho, fp64=True)
    assert np.all(rel_errors(got, ref, comps) <= TOL64)
    r = np.random.default_rng(comps).normal(size=ref.shape)
    ga = run_adjoint(mesh.tuple(), comps, r, True)
    gr = orc.adjoint(mesh.tuple(), comps, r)
    assert np.linalg.norm(ga - gr) <= TOL64 * np.linalg.norm(gr)


def test_paper_cube_model(gravlib, orc):
    """Sec. 3.1 (tests/golden/sec3_1_cube_model.txt): a 300 m cube 500-800 m
    deep (+300 kg/m^3) under 40x40 stations at 50 m spacing, 50 m up.  The
    paper reads its fast forward's residual 13 orders of magnitude below the
    field off Figs. 6 and 7; the FP64 path here agrees with the exact
    single-prism field to one order of that (relative L2 per component)."""
    claim = golden_data.load("sec3_1_cube_model.txt")["residual_orders"]
    mesh, rho, boxes = W.cube40()
    got = run_forward(mesh.tuple(), ALL7, rho, fp64=True)
    l0, l1, m0, m1, n0, n1, d = boxes[0]
    ref = orc.box_field(mesh.tuple(), ALL7, (l0, l1, m0, m1, n0, n1), d).reshape(7, mesh.ny, mesh.nx)
    err = rel_errors(got, ref, ALL7)
    assert np.all(err <= 10.0 ** (1 - claim)), err
    got32 = run_forward(mesh.tuple(), ALL7, rho.astype(np.float32), fp64=False)
    assert np.all(rel_errors(got32, ref, ALL7) <= TOL32)
    # element-wise, in mGal (gz) and Eotvos (gradients), against each component's
    # peak over the 40 x 40 stations: FP64 1e-10, FP32 2e-5 (the bounds of the
    # full-size tests)
    units = np.array([1e5] + [1e9] * 6)[:, None]
    peak = np.abs(ref.reshape(7, -1) * units).max(axis=1)
    max64 = np.abs((got - ref).reshape(7, -1) * units).max(axis=1)
    max32 = np.abs((got32 - ref).reshape(7, -1) * units).max(axis=1)
    print("cube max abs FP64", max64, "FP32", max32, "peak", peak)
    assert np.all(max64 <= 1e-10 * peak), (max64, peak)
    assert np.all(max32 <= 2e-5 * peak), (max32, peak)


def test_boxes256_fp64_vs_oracle_and_superposition(gravlib, orc):
    """256x256x32 mesh of 20 random boxes plus noise: sampled stations
    against direct summation; the noise-free field against the sum of the
    boxes' closed forms at every station."""
    mesh, rho, boxes = W.boxes256()
    comps = ALL7
    got = run_forward(mesh.tuple(), comps, rho, fp64=True)
    st = W.station_subset(mesh, 24, np.random.default_rng(5))
    ref = orc.forward(mesh.tuple(), comps, rho, stations=st)
    err = rel_errors(got.reshape(7, -1)[:, st], ref, comps)
    assert np.all(err <= TOL64), err

    _, rho_clean, _ = W.boxes256(noise=False)
    got_clean = run_forward(mesh.tuple(), comps, rho_clean, fp64=True)
    st2 = np.arange(0, mesh.nx * mesh.ny, 97, dtype=np.int64)
    ref2 = sum(orc.box_field(mesh.tuple(), comps, b[:6], b[6], stations=st2) for b in boxes)
    err2 = rel_errors(got_clean.reshape(7, -1)[:, st2], ref2, comps)
    assert np.all(err2 <= TOL64), err2


@pytest.mark.parametrize("mesh", [(45, 23, 7, 20.0, 25.0, 10.0, 3.0),     # 64-point columns
                                  (21, 300, 11, 20.0, 15.0, 10.0, 3.0),   # 512-point, two per warp
                                  (9, 600, 10, 20.0, 15.0, 10.0, 3.0)])   # 1024-point warp transforms
def test_dot_product_adjoint(gravlib, mesh):
    """<G x, y> = <x, G^T y> on ragged meshes, FP64 and FP32."""
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(11)
    x = rng.normal(size=(nz, ny, nx))
    y = rng.normal(size=(7, ny, nx))
    for fp64, tol in ((True, 1e-12), (False, 1e-5)):
        dt = torch.float64 if fp64 else torch.float32
        with Plan(mesh, ALL7, fp64=fp64) as plan:
            xt = torch.as_tensor(x, dtype=dt).cuda()
            yt = torch.as_tensor(y, dtype=dt).cuda()
            gx = plan.forward(xt).double()
            gty = plan.adjoint(yt).double()
            lhs = float((gx * yt.double()).sum())
            rhs = float((xt.double() * gty).sum())
        assert abs(lhs - rhs) <= tol * max(abs(lhs), abs(rhs)), (fp64, lhs, rhs)


# Meshes with 513 <= ny <= 1024: Py = 2048, so the FP32 forward runs the
# 1024-point column kernel with one warp per layer transform (ragged ny_pad,
# fewer layers than FFT warps, and enough layers to wrap every ring).
WIDE_MESHES = [
    (3, 1024, 20, 10.0, 10.0, 10.0, 2.0),
    (5, 513, 9, 20.0, 15.0, 10.0, 3.0),
    (2, 700, 1, 10.0, 10.0, 10.0, 1.0),
]


def check_fp32_columns(orc, mesh, comps):
    """FP32 forward against the oracle at sampled stations and against the
    FP64 spectral path at every station; the FP32 adjoint against the FP64
    adjoint at every cell."""
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 1000 + ny + nz)
    rho = rng.uniform(-300, 300, (nz, ny, nx))
    got32 = run_forward(mesh, comps, rho, fp64=False).reshape(len(capi.comp_list(comps)), -1)
    got64 = run_forward(mesh, comps, rho, fp64=True).reshape(len(capi.comp_list(comps)), -1)
    st = np.unique(np.concatenate([[0, nx * ny - 1, nx * (ny // 2)],
                                   rng.integers(0, nx * ny, 29)])).astype(np.int32)
    ref = orc.forward(mesh, comps, rho, stations=st)
    assert np.all(rel_errors(got32[:, st], ref, comps) <= TOL32)
    assert np.all(rel_errors(got64[:, st], ref, comps) <= TOL64)
    assert np.all(rel_errors(got32, got64, comps) <= TOL32)
    r = rng.normal(size=(len(capi.comp_list(comps)), ny, nx))
    g32 = run_adjoint(mesh, comps, r, fp64=False).reshape(-1)
    g64 = run_adjoint(mesh, comps, r, fp64=True).reshape(-1)
    assert np.linalg.norm(g32 - g64) <= TOL32 * np.linalg.norm(g64)


@pytest.mark.parametrize("mesh", WIDE_MESHES)
@pytest.mark.parametrize("comps", [ALL7, 0x3F, capi.GRAV_GZ, capi.GRAV_GXY | capi.GRAV_GYZ, ALL7_GXY_SANS_GZZ])
def test_forward_fp32_wide_columns(gravlib, orc, mesh, comps):
    """2048-point columns (1024-point warp transforms): forward and adjoint."""
    check_fp32_columns(orc, mesh, comps)


# Meshes with 257 <= ny <= 512: Py = 1024, so the FP32 forward runs the
# 512-point column kernel with both ky parities in one CTA and two transforms
# per warp (ragged ny_pad, fewer layers than FFT warps, enough layers to wrap
# every ring and cross a compensated block); eight components take the
# fallback kernel.
MID_MESHES = [
    (3, 512, 20, 10.0, 10.0, 10.0, 2.0),
    (5, 257, 9, 20.0, 15.0, 10.0, 3.0),
    (2, 300, 1, 10.0, 10.0, 10.0, 1.0),
    (33, 420, 40, 20.0, 20.0, 15.0, 4.0),
]


@pytest.mark.parametrize("mesh", MID_MESHES)
@pytest.mark.parametrize("comps", [ALL7, 0x3F, capi.GRAV_GZ, capi.GRAV_GXY | capi.GRAV_GYZ, ALL7_GXY_SANS_GZZ])
def test_forward_fp32_mid_columns(gravlib, orc, mesh, comps):
    """1024-point columns (512-point transforms, two per warp): forward and adjoint."""
    check_fp32_columns(orc, mesh, comps)


# Meshes with 513 <= nx <= 1024: Px = 2048, so the FP32 row stages run the
# split even/odd warp transforms with staged rows (nx a multiple of 4) or the
# block transform (nx = 513); ragged row counts included.
WIDE_ROW_MESHES = [
    (600, 3, 4, 10.0, 10.0, 10.0, 2.0),
    (1024, 2, 3, 10.0, 12.0, 10.0, 1.0),
    (516, 9, 11, 20.0, 15.0, 10.0, 3.0),
    (513, 7, 2, 20.0, 15.0, 10.0, 3.0),
]


@pytest.mark.parametrize("mesh", WIDE_ROW_MESHES)
def test_fp32_wide_rows(gravlib, orc, mesh):
    """FP32 forward and adjoint on 2048-point rows: against the oracle at
    sampled stations, and against the FP64 spectral path everywhere."""
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx + 7 * ny + nz)
    rho = rng.uniform(-300, 300, (nz, ny, nx))
    got32 = run_forward(mesh, ALL7, rho, fp64=False).reshape(7, -1)
    got64 = run_forward(mesh, ALL7, rho, fp64=True).reshape(7, -1)
    st = np.unique(np.concatenate([[0, nx * ny - 1, nx // 2], rng.integers(0, nx * ny, 21)])).astype(np.int32)
    ref = orc.forward(mesh, ALL7, rho, stations=st)
    assert np.all(rel_errors(got32[:, st], ref, ALL7) <= TOL32)
    assert np.all(rel_errors(got32, got64, ALL7) <= TOL32)
    r = rng.normal(size=(7, ny, nx))
    g32 = run_adjoint(mesh, ALL7, r, fp64=False).reshape(-1)
    g64 = run_adjoint(mesh, ALL7, r, fp64=True).reshape(-1)
    assert np.linalg.norm(g32 - g64) <= TOL32 * np.linalg.norm(g64)


# Both axes 513..1024 (Px = Py = 2048) with ny a multiple of 4 and 8:
# the FP32 adjoint writes its column output tile-major and reads it back
# by whole tiles (the last tile ragged for ny = 517).
WIDE_BOTH_MESHES = [
    (520, 600, 5, 20.0, 20.0, 10.0, 4.0),
    (600, 517, 3, 10.0, 10.0, 10.0, 2.0),
]


@pytest.mark.parametrize("mesh", WIDE_BOTH_MESHES)
def test_fp32_adjoint_wide_both(gravlib, mesh):
    """FP32 adjoint against the FP64 adjoint at every cell, and the FP32
    dot-product identity <G x, y> = <x, G^T y>."""
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 3 + ny)
    r = rng.normal(size=(7, ny, nx))
    g32 = run_adjoint(mesh, ALL7, r, fp64=False)
    g64 = run_adjoint(mesh, ALL7, r, fp64=True)
    assert np.linalg.norm((g32 - g64).ravel()) <= TOL32 * np.linalg.norm(g64.ravel())
    x = rng.uniform(-300, 300, (nz, ny, nx))
    gx = run_forward(mesh, ALL7, x, fp64=False).astype(np.float64)
    lhs = float(np.dot(gx.ravel(), r.ravel()))
    rhs = float(np.dot(x.ravel(), g32.astype(np.float64).ravel()))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(gx.ravel()) * np.linalg.norm(r.ravel())


@pytest.mark.parametrize("mesh", [SMALL_MESHES[0], SMALL_MESHES[3], SMALL_MESHES[5], (64, 1, 3, 10.0, 10.0, 10.0, 2.0)])
@pytest.mark.parametrize("comps", [capi.GRAV_GX | capi.GRAV_GY, ALL7_GXY_SANS_GZZ,
                                   capi.GRAV_GZ | capi.GRAV_GX | capi.GRAV_GZZ])
def test_first_derivatives_match_oracle(gravlib, orc, mesh, comps):
    """gx, gy (alone and with the other components) through the whole path:
    FP64 and FP32 forward and adjoint against the oracle."""
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(nx * 7 + ny + comps)
    rho = rng.uniform(-500, 500, (nz, ny, nx))
    ref = orc.forward(mesh, comps, rho)
    assert np.all(rel_errors(run_forward(mesh, comps, rho, fp64=True), ref, comps) <= TOL64)
    assert np.all(rel_errors(run_forward(mesh, comps, rho.astype(np.float32), fp64=False), ref, comps) <= TOL32)
    r = rng.normal(size=(len(capi.comp_list(comps)), ny, nx))
    gref = orc.adjoint(mesh, comps, r)
    for fp64, tol in ((True, TOL64), (False, TOL32)):
        g = run_adjoint(mesh, comps, r, fp64=fp64)
        assert np.linalg.norm(g - gref) <= tol * np.linalg.norm(gref), fp64


def test_repeatable_and_stream_ordered(gravlib):
    """Two calls give bit-identical results, on a non-default stream too."""
    mesh, rho = W.small16()
    with Plan(mesh, ALL7) as plan:
        x = torch.as_tensor(rho, dtype=torch.float32).cuda()
        a = plan.forward(x).clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b = plan.forward(x, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_max_size_axes(gravlib, orc):
    """Largest axes the plan accepts (nx = 2048 with ny small, ny = 1024 with
    nx small), against the oracle at a few stations."""
    for mesh in [(capi.GRAV_MAX_NX, 2, 1, 10.0, 10.0, 10.0, 5.0), (3, capi.GRAV_MAX_NY, 1, 10.0, 10.0, 10.0, 5.0)]:
        nx, ny, nz = mesh[:3]
        rho = np.random.default_rng(nx + ny).uniform(-300, 300, (nz, ny, nx))
        got = run_forward(mesh, ALL7, rho, fp64=True)
        st = np.array([0, nx * ny - 1, (ny // 2) * nx + nx // 2, 1, nx * ny // 3], dtype=np.int32)
        ref = orc.forward(mesh, ALL7, rho, stations=st)
        assert np.all(rel_errors(got.reshape(7, -1)[:, st], ref, ALL7) <= TOL64)
