"""Pins of the oracle's equal-dimension variant (Sec. 2.2, Eqs. 10-11: a
station at the centre of every cell, data as three-dimensional as the mesh)
against things other than itself: the block-Toeplitz structure in all three
offsets, reduction to the already pinned observation-plane oracle for the
cells below a station and, mirrored, for the cells above it, Poisson's
equation inside a uniform mesh, and the exact field at a cube's centre."""
import numpy as np
import pytest

import oracle

ALL9 = 0x1FF
UPS = 6.672e-11
Z_ODD = [0, 3, 5]  # gz, gxz, gyz change sign under z -> -z; the others do not


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def test_forward_equals_explicit_G():
    mesh = (4, 3, 3, 10.0, 12.0, 8.0, 1.0)
    rho = np.random.default_rng(1).uniform(-300, 300, (3, 3, 4))
    G = oracle.gmatrix3d(mesh, ALL9)
    d = oracle.forward3d(mesh, ALL9, rho)
    assert np.allclose(d.reshape(9, -1), np.einsum("cij,j->ci", G, rho.reshape(-1)), rtol=1e-13, atol=0)


def test_adjoint_is_the_transpose():
    """adjoint3d equals the explicit G transposed, and <G x, r> = <x, G^T r>
    holds on a larger mesh without the explicit G."""
    mesh = (4, 3, 3, 10.0, 12.0, 8.0, 1.0)
    rng = np.random.default_rng(6)
    r = rng.normal(size=(9, 3, 3, 4))
    G = oracle.gmatrix3d(mesh, ALL9)
    got = oracle.adjoint3d(mesh, ALL9, r).reshape(-1)
    want = np.einsum("cij,ci->j", G, r.reshape(9, -1))
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    mesh = (7, 6, 5, 10.0, 12.0, 8.0, 1.0)
    x = rng.normal(size=(5, 6, 7))
    r = rng.normal(size=(9, 5, 6, 7))
    lhs = float((oracle.forward3d(mesh, ALL9, x) * r).sum())
    rhs = float((x * oracle.adjoint3d(mesh, ALL9, r)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_three_level_toeplitz():
    """G depends only on the offsets (l - p, m - q, n - t) (Eq. 10 in all
    three axes): (2nx - 1)(2ny - 1)(2nz - 1) values per component, the count
    of Eq. 11 without the virtual grid's extra row."""
    nx, ny, nz = 4, 3, 3
    mesh = (nx, ny, nz, 10.0, 12.0, 8.0, 1.0)
    G = oracle.gmatrix3d(mesh, ALL9)
    idx = np.arange(nx * ny * nz)
    p, q, t = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    off = {}
    for i in idx:
        for j in idx:
            key = (p[j] - p[i], q[j] - q[i], t[j] - t[i])
            off.setdefault(key, []).append((i, j))
    assert len(off) == (2 * nx - 1) * (2 * ny - 1) * (2 * nz - 1)
    scale = np.abs(G).max(axis=(1, 2))
    for pairs in off.values():
        vals = np.array([G[:, i, j] for i, j in pairs])
        assert np.all(np.abs(vals - vals[0]) <= 1e-12 * scale)


@pytest.mark.parametrize("t", [0, 2])
def test_cells_below_the_station_reduce_to_the_plane_oracle(t):
    """With density only in the layers below station layer t, the field at
    (p, q, t) is the observation-plane forward of those layers with the
    stations dz / 2 above their top."""
    nx, ny, nz, dx, dy, dz = 5, 4, 5, 10.0, 12.0, 8.0
    rho = np.random.default_rng(2 + t).uniform(-300, 300, (nz, ny, nx))
    rho[: t + 1] = 0.0
    d3 = oracle.forward3d((nx, ny, nz, dx, dy, dz, 1.0), ALL9, rho)[:, t]
    d2 = oracle.forward((nx, ny, nz - t - 1, dx, dy, dz, dz / 2), ALL9, rho[t + 1:])
    assert np.allclose(d3, d2, rtol=1e-12, atol=1e-12 * np.abs(d2).max())


@pytest.mark.parametrize("t", [2, 4])
def test_cells_above_the_station_are_the_mirrored_plane_oracle(t):
    """Density only above station layer t: reflecting z about the station's
    depth maps those layers onto a mesh below a plane dz / 2 above it, so the
    field is the plane forward of the reversed layers with the components
    odd in z negated."""
    nx, ny, nz, dx, dy, dz = 5, 4, 5, 10.0, 12.0, 8.0
    rho = np.random.default_rng(7 + t).uniform(-300, 300, (nz, ny, nx))
    rho[t:] = 0.0
    d3 = oracle.forward3d((nx, ny, nz, dx, dy, dz, 1.0), ALL9, rho)[:, t]
    d2 = oracle.forward((nx, ny, t, dx, dy, dz, dz / 2), ALL9, rho[:t][::-1])
    d2[Z_ODD] *= -1.0
    assert np.allclose(d3, d2, rtol=1e-12, atol=1e-12 * np.abs(d2).max())


def test_uniform_mesh_obeys_poisson():
    """A uniform density rho0 everywhere: every station is inside the body,
    so the trace of the gradient tensor is -4 pi upsilon rho0 at each."""
    mesh = (5, 4, 3, 10.0, 12.0, 8.0, 1.0)
    rho0 = 250.0
    d = oracle.forward3d(mesh, 0x52, np.full((3, 4, 5), rho0))  # gxx, gyy, gzz
    trace = d.sum(axis=0)
    assert np.allclose(trace, -4 * np.pi * UPS * rho0, rtol=1e-12, atol=0)


def test_own_cell_of_a_cube_mesh():
    """Only the station's own cell (a cube) carries density: the odd
    components vanish there and each diagonal one is -4 pi upsilon rho / 3."""
    nx, ny, nz = 3, 3, 3
    rho = np.zeros((nz, ny, nx))
    rho[1, 1, 1] = 300.0
    d = oracle.forward3d((nx, ny, nz, 10.0, 10.0, 10.0, 1.0), ALL9, rho)[:, 1, 1, 1]
    assert np.allclose(d[[0, 2, 3, 5, 7, 8]], 0.0, atol=1e-14 * 4 * np.pi * UPS * 300.0)
    assert np.allclose(d[[1, 4, 6]], -4 * np.pi * UPS * 300.0 / 3, rtol=1e-13)


def test_three_level_circulant_spectra_are_real_or_imaginary():
    """The structure a transform-based equal-dimension path relies on, from
    the oracle's explicit G: embedded in a three-level circulant (negative
    offsets wrapped), each component's kernel has a purely real or purely
    imaginary spectrum (gz, gx, gy imaginary; gxx, gxy, gxz, gyy, gyz, gzz
    real: odd in an odd number of axes), and the circulant product equals
    the direct sum."""
    nx, ny, nz = 5, 4, 3
    mesh = (nx, ny, nz, 10.0, 12.0, 8.0, 1.0)
    G = oracle.gmatrix3d(mesh, ALL9)
    rho = np.random.default_rng(4).normal(size=(nz, ny, nx))
    ref = oracle.forward3d(mesh, ALL9, rho)
    Px, Py, Pz = 16, 8, 8  # powers of two >= 2n - 1 (9, 7, 5)
    i = np.arange(nx * ny * nz)
    p, q, t = i % nx, (i // nx) % ny, i // (nx * ny)
    R = np.zeros((Pz, Py, Px))
    R[:nz, :ny, :nx] = rho
    imaginary = {0, 7, 8}
    for c in range(9):
        K = np.zeros((Pz, Py, Px))
        # d(i) = sum_j K(j - i) rho(j): K(-offset) stored at offset mod P (a circular convolution)
        K[(t[:, None] - t[None, :]) % Pz, (q[:, None] - q[None, :]) % Py, (p[:, None] - p[None, :]) % Px] = G[c]
        S = np.fft.fftn(K)
        small = (np.abs(S.real) if c in imaginary else np.abs(S.imag)).max()
        assert small <= 1e-12 * np.abs(S).max(), c
        d = np.real(np.fft.ifftn(S * np.fft.fftn(R)))[:nz, :ny, :nx]
        assert np.abs(d - ref[c]).max() <= 1e-12 * np.abs(ref[c]).max(), c


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.forward3d((0, 2, 2, 1.0, 1.0, 1.0, 1.0), 1, np.zeros(0))
    with pytest.raises(ValueError):
        oracle.forward3d((2, 2, 2, 1.0, 1.0, 1.0, 1.0), 1, np.zeros((2, 2, 2)), stations=[8])


# Planted mistakes in the equal-dimension code of the oracle's C source; each
# must fail the reduction pins above (built and run the same way as
# tests/test_oracle_mutants.py does for the plane oracle).
MUTANTS_3D = {
    "station_depth_at_cell_bottom": ("z = (t + 0.5) * g->dz", "z = (t + 1.0) * g->dz"),
    "station_layer_index": ("t = st / (g->nx * g->ny)", "t = st / g->nx % g->nz"),
    "station_y_uses_dx": ("y = (q + 0.5) * g->dy, z = (t + 0.5)", "y = (q + 0.5) * g->dx, z = (t + 0.5)"),
}


def _build_lib(tmp_path, name, old, new):
    import ctypes
    import os
    import subprocess

    src = open(os.path.join(os.path.dirname(oracle.__file__), "prism_oracle.c")).read()
    assert src.count(old) == 1, name
    c_path, so_path = tmp_path / f"{name}.c", tmp_path / f"{name}.so"
    c_path.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so_path), str(c_path), "-lm",
                    "-lpthread"], check=True)
    lib = ctypes.CDLL(str(so_path))
    d, i, u, p = ctypes.c_double, ctypes.c_int, ctypes.c_uint, ctypes.c_void_p
    lib.orc_forward.argtypes = [i, i, i, d, d, d, d, u, p, i, p, p, i]
    lib.orc_forward3d.argtypes = [i, i, i, d, d, d, u, p, i, p, p, i]
    return lib


def _reductions_hold(lib):
    """The below- and above-the-station reductions of the pins, run on lib."""
    import ctypes

    nx, ny, nz, dx, dy, dz = 4, 3, 5, 10.0, 12.0, 8.0
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    for t, below in ((1, True), (3, False)):
        rho = np.random.default_rng(t).uniform(-300, 300, (nz, ny, nx))
        if below:
            rho[: t + 1] = 0.0
            sub = np.ascontiguousarray(rho[t + 1:])
        else:
            rho[t:] = 0.0
            sub = np.ascontiguousarray(rho[:t][::-1])
        st3 = (np.arange(nx * ny) + t * nx * ny).astype(np.int32)
        d3 = np.zeros((9, nx * ny))
        lib.orc_forward3d(nx, ny, nz, dx, dy, dz, ALL9, ptr(rho), nx * ny, ptr(st3), ptr(d3), 1)
        st2 = np.arange(nx * ny, dtype=np.int32)
        d2 = np.zeros((9, nx * ny))
        lib.orc_forward(nx, ny, sub.shape[0], dx, dy, dz, dz / 2, ALL9, ptr(sub), nx * ny, ptr(st2), ptr(d2), 1)
        if not below:
            d2[Z_ODD] *= -1.0
        if not np.allclose(d3, d2, rtol=1e-10, atol=1e-10 * np.abs(d2).max()):
            return False
    return True


def test_unmutated_equal_dim_code_passes(tmp_path):
    assert _reductions_hold(_build_lib(tmp_path, "original", "#include <math.h>", "#include <math.h>"))


@pytest.mark.parametrize("name", sorted(MUTANTS_3D))
def test_equal_dim_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS_3D[name]
    assert not _reductions_hold(_build_lib(tmp_path, name, old, new)), f"planted mistake {name} was not caught"
