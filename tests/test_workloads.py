"""The seeded synthetic inputs follow their stated recipes: the same seed
gives the same data, boxes lie inside the mesh with the stated extents and
values, the Gaussian random field has the stated mean, standard deviation and
correlation length, and the Sec. 3.1 cube sits where the paper puts it."""
import numpy as np
import pytest

import golden_data
from paper_2005_10160_gb300 import workloads as W


def test_generators_are_deterministic():
    for make in (W.small16, W.boxes256, W.boxes512, W.cube40):
        a, b = make(), make()
        assert a[0] == b[0]
        assert np.array_equal(a[1], b[1])


def test_random_boxes_inside_the_mesh_with_stated_extents():
    mesh = W.Mesh(40, 24, 12, 10.0, 10.0, 10.0, 1.0)
    boxes = W.random_boxes(mesh, 500, W.rng_for(7), 300.0)
    for (l0, l1, m0, m1, n0, n1, d) in boxes:
        for lo, hi, n in ((l0, l1, mesh.nx), (m0, m1, mesh.ny), (n0, n1, mesh.nz)):
            assert 0 <= lo < hi <= n
            assert hi - lo <= max(1, n // 4)
        assert d in (300.0, -300.0)
    signs = np.array([b[6] for b in boxes])
    assert 0.4 < (signs > 0).mean() < 0.6  # the sign is a fair draw


def test_paint_boxes_superposes():
    mesh = W.Mesh(8, 6, 4, 1.0, 1.0, 1.0, 1.0)
    boxes = [(0, 4, 0, 3, 0, 2, 10.0), (2, 6, 1, 5, 1, 4, -4.0)]
    rho = W.paint_boxes(mesh, boxes)
    assert rho.shape == (4, 6, 8)
    assert rho[1, 2, 3] == 6.0 and rho[0, 0, 0] == 10.0 and rho[3, 4, 5] == -4.0 and rho[3, 0, 7] == 0.0
    assert rho.sum() == 10.0 * 4 * 3 * 2 - 4.0 * 4 * 4 * 3


def test_boxes512_has_the_three_stated_densities():
    mesh, rho, boxes = W.boxes512()
    assert mesh.tuple() == (512, 512, 64, 20.0, 20.0, 20.0, 10.0)
    assert [b[6] for b in boxes] == [400.0, -300.0, 250.0]
    assert rho.shape == (64, 512, 512)


def test_random_field_moments_and_correlation_length():
    """White N(0,1) noise filtered by a Gaussian of std l / sqrt(2) cells has
    correlation exp(-lag^2 / (2 l^2)): e^(-1/2) at lag l along every axis."""
    torch = pytest.importorskip("torch")
    ell = 6.0
    mesh, f = W.grf1024(nx=96, ny=80, nz=48, corr_cells=ell, std=200.0)
    assert mesh.tuple()[:3] == (96, 80, 48) and f.dtype == torch.float32
    x = f.double().numpy()
    assert abs(x.mean()) < 1e-3 and abs(x.std() - 200.0) < 1e-2
    lag = int(ell)
    for axis in range(3):
        c = (x * np.roll(x, lag, axis=axis)).mean() / x.var()  # periodic field
        assert abs(c - np.exp(-0.5)) < 0.1, (axis, c)


def test_cube40_is_the_sec31_model():
    """The model as Sec. 3.1 prints it (tests/golden/sec3_1_cube_model.txt):
    300 m cube, top 500 m and bottom 800 m below the ground, +300 kg/m^3,
    centred under the middle of the 40 x 40 station grid (50 m spacing), with
    the stations 50 m above the ground, on 40 x 40 x 20 = 32000 cells."""
    g = golden_data.load("sec3_1_cube_model.txt")
    mesh, rho, [box] = W.cube40()
    l0, l1, m0, m1, n0, n1, d = box
    assert (mesh.nx, mesh.ny, mesh.nz) == (g["mesh_nx"], g["mesh_ny"], g["mesh_nz"])
    assert mesh.nx * mesh.ny * mesh.nz == g["cells"]
    assert (mesh.nx, mesh.ny) == (g["stations_x"], g["stations_y"]) and mesh.nx * mesh.ny == g["stations"]
    assert (mesh.dx, mesh.dy, mesh.h) == (g["station_spacing"], g["station_spacing"], g["station_height"])
    side = g["cube_size"]
    assert ((l1 - l0) * mesh.dx, (m1 - m0) * mesh.dy, (n1 - n0) * mesh.dz) == (side, side, side)
    assert (n0 * mesh.dz, n1 * mesh.dz, d) == (g["cube_top"], g["cube_bottom"], g["cube_density"])
    assert mesh.nz * mesh.dz >= g["cube_bottom"]
    centre = 0.5 * mesh.nx * mesh.dx  # middle of the stations (p + 1/2) dx, p < 40
    assert 0.5 * (l0 + l1) * mesh.dx == centre and 0.5 * (m0 + m1) * mesh.dy == centre
    assert np.count_nonzero(rho) == (side / mesh.dx) ** 3


def test_station_subset_holds_corners_and_centre():
    mesh = W.Mesh(37, 29, 3, 1.0, 1.0, 1.0, 1.0)
    st = W.station_subset(mesh, 20, W.rng_for(5))
    assert len(st) == 20 and len(set(st.tolist())) == 20
    assert {0, 36, 28 * 37, 29 * 37 - 1, 14 * 37 + 18} <= set(st.tolist())
    assert st.min() >= 0 and st.max() < 37 * 29
