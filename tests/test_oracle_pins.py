"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against an independent fact: brute-force
quadrature of the Newtonian integrals, the far-field point mass, the Bouguer
slab value 2 pi upsilon rho dz, the Laplace trace of the gradient tensor
(Eq. 1), finite differences of gz, the parity of the kernel under
reflection, translation invariance (Eq. 7) and superposition over cells
(Eq. 3).  A dropped term, a wrong sign, a swapped axis or a wrong cell index
in the oracle fails at least one of them.
"""
import numpy as np
import pytest

import golden_data
from quadrature import point_mass, prism_quadrature
from paper_2005_10160_gb300 import workloads as W

ALL7 = 0x7F


@pytest.mark.parametrize(
    "station,box",
    [
        ((5.0, 5.0, -1.0), (0.0, 10.0, 0.0, 10.0, 0.0, 10.0)),    # just above the centre
        ((13.0, -4.0, -7.0), (0.0, 10.0, 0.0, 20.0, 0.0, 15.0)),  # off to one side
        ((2.0, 30.0, -3.0), (0.0, 10.0, 0.0, 20.0, 0.0, 15.0)),
        ((-6.0, 11.0, -2.5), (-3.0, 4.0, 5.0, 9.0, 1.0, 2.0)),    # thin layer
    ],
)
def test_closed_forms_match_quadrature(orc, station, box):
    """All nine closed forms (Eq. 2, the gradient forms and the horizontal
    first derivatives) equal brute-force Gauss-Legendre quadrature of the
    volume integrals."""
    ref = prism_quadrature(station, box, nsub=8, order=16)
    got = orc.prism(station, box)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale, (got - ref) / scale


@pytest.mark.parametrize("station", [(0.0, 0.0, -50.0), (975.0, -975.0, -50.0), (-525.0, 275.0, -50.0),
                                     (150.0, 0.0, -50.0)])
def test_paper_cube_matches_quadrature(orc, station):
    """The test model of Sec. 3.1 at its own scale: a 300 m cube centred under
    the origin, top 500 m and bottom 800 m below the ground, observed 50 m above
    the ground at stations of the 50 m grid (centre, far corner, off-axis, above
    an edge).  The nine closed forms equal quadrature to 1e-12, first and second
    derivatives each relative to their own largest value (their units differ by
    a length).  The paper reports its fast algorithm 13 orders of magnitude
    below the fields it computes, so the reference it is compared with must be
    exact to well beyond that."""
    g = golden_data.load("sec3_1_cube_model.txt")
    half = 0.5 * g["cube_size"]
    box = (-half, half, -half, half, g["cube_top"], g["cube_bottom"])
    assert station[2] == -g["station_height"]
    ref = prism_quadrature(station, box, nsub=8, order=16)
    got = orc.prism(station, box)
    first, second = [0, 7, 8], [1, 2, 3, 4, 5, 6]
    for idx in (first, second):
        scale = np.abs(ref[idx]).max()
        assert np.abs(got[idx] - ref[idx]).max() <= 1e-12 * scale, (idx, (got[idx] - ref[idx]) / scale)


@pytest.mark.parametrize("station", [(25.0, 5.0, 5.0), (-12.0, 17.0, 3.0), (15.0, 15.0, 9.0), (5.0, 25.0, 0.5),
                                     (30.0, -7.0, 12.0)])
def test_closed_forms_hold_level_with_the_prism(orc, station):
    """Stations beside the prism at depths inside its depth range (corners
    on both sides of the station's z, where the atan terms change branch):
    all nine closed forms still equal quadrature to 1e-12."""
    box = (0.0, 10.0, 0.0, 10.0, 0.0, 10.0)
    ref = prism_quadrature(station, box, nsub=8, order=16)
    got = orc.prism(station, box)
    for idx in ([0, 7, 8], [1, 2, 3, 4, 5, 6]):
        scale = np.abs(ref[idx]).max()
        assert np.abs(got[idx] - ref[idx]).max() <= 1e-12 * scale, (idx, (got[idx] - ref[idx]) / scale)


@pytest.mark.parametrize("box", [(0.0, 10.0, 0.0, 10.0, 0.0, 10.0), (0.0, 20.0, 0.0, 12.0, 0.0, 7.0),
                                 (-3.0, 4.0, 5.0, 9.0, 1.0, 2.5)])
@pytest.mark.parametrize("frac", [(0.5, 0.5, 0.5), (0.2, 0.7, 0.4), (0.9, 0.1, 0.65), (0.33, 0.5, 0.95)])
def test_interior_points_obey_poisson(orc, box, frac):
    """Stations inside the prism (quadrature does not apply: the integrand
    is singular there): the trace of the gradient tensor is -4 pi upsilon rho
    (Poisson's equation instead of Laplace's), and the derivatives of gz by
    fourth-order finite differences equal gxz, gyz and gzz."""
    st = np.array([box[2 * i] + frac[i] * (box[2 * i + 1] - box[2 * i]) for i in range(3)])
    g = orc.prism(tuple(st), box) / 6.672e-11  # per unit upsilon rho
    assert abs(g[1] + g[4] + g[6] + 4 * np.pi) <= 1e-12 * 4 * np.pi
    h = 1e-3 * min(box[1] - box[0], box[3] - box[2], box[5] - box[4])

    def gz(p):
        return orc.prism(tuple(p), box)[0] / 6.672e-11

    for axis, comp in ((0, 3), (1, 5), (2, 6)):
        e = np.zeros(3)
        e[axis] = h
        fd = (-gz(st + 2 * e) + 8 * gz(st + e) - 8 * gz(st - e) + gz(st - 2 * e)) / (12 * h)
        assert abs(fd - g[comp]) <= 1e-9 * 4 * np.pi, (axis, fd, g[comp])


def test_cube_centre_field(orc):
    """At the centre of a cube every odd component vanishes and each diagonal
    component is a third of -4 pi upsilon rho."""
    g = orc.prism((5.0, 5.0, 5.0), (0.0, 10.0, 0.0, 10.0, 0.0, 10.0)) / 6.672e-11
    assert np.allclose(g[[0, 2, 3, 5, 7, 8]], 0.0, atol=1e-13)
    assert np.allclose(g[[1, 4, 6]], -4 * np.pi / 3, rtol=1e-13)


@pytest.mark.parametrize("direction", [(1, 0.3, 2), (-2, 1, 1), (0.2, -0.1, 3), (3, 3, 0.5)])
def test_far_field_point_mass_cube(orc, direction):
    """A cube has no quadrupole moment, so far away it acts as a point mass
    with relative error O((a/R)^4)."""
    a = 10.0
    box = (0.0, a, 0.0, a, 100.0, 100.0 + a)
    centre = np.array([a / 2, a / 2, 100.0 + a / 2])
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    R = 400.0  # far enough for the multipole bound, near enough that the
    # FP64 cancellation of the eight corner terms stays far below (a/R)^4
    station = centre - R * d
    got = orc.prism(station, box)
    ref = point_mass(station, centre, a ** 3)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 5 * (a / R) ** 4 * scale


def test_far_field_point_mass_general_prism(orc):
    """A general prism: the leading error is the quadrupole, O((a/R)^2)."""
    box = (0.0, 10.0, 0.0, 30.0, 50.0, 55.0)
    centre = np.array([5.0, 15.0, 52.5])
    station = centre + np.array([-900.0, 400.0, -1500.0])
    R = np.linalg.norm(centre - station)
    got = orc.prism(station, box)
    ref = point_mass(station, centre, 10.0 * 30.0 * 5.0)
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    assert err <= 2 * (30.0 / R) ** 2
    assert err > 1e-12  # the quadrupole term is really there


def test_bouguer_slab(orc):
    """A wide thin slab gives 2 pi upsilon rho dz, with relative error about
    (2h + dz) / (2L); the gradient of an infinite slab is zero."""
    L, dz, h = 1.0e6, 10.0, 1.0
    box = (-L, L, -L, L, 0.0, dz)
    got = orc.prism((0.0, 0.0, -h), box)
    bouguer = 2 * np.pi * 6.672e-11 * dz
    assert abs(got[0] - bouguer) <= 2 * (2 * h + dz) / (2 * L) * bouguer
    assert abs(got[0] - bouguer) > 0  # finite slab, not the infinite one
    for c in (1, 4, 6):
        assert abs(got[c]) <= 1e-4 * bouguer / dz


@pytest.mark.parametrize("seed", range(5))
def test_laplace_trace(orc, seed):
    """The gradient tensor is trace free: gxx + gyy + gzz = 0 (Eq. 1)."""
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-20, 20, 3)
    ext = rng.uniform(1, 30, 3)
    lo[2] = abs(lo[2])
    box = (lo[0], lo[0] + ext[0], lo[1], lo[1] + ext[1], lo[2], lo[2] + ext[2])
    station = (rng.uniform(-40, 40), rng.uniform(-40, 40), -rng.uniform(0.5, 20))
    g = orc.prism(station, box)
    scale = np.abs(g[1:]).max()
    assert abs(g[1] + g[4] + g[6]) <= 1e-13 * scale


@pytest.mark.parametrize("station", [(3.0, 4.0, -2.0), (-12.0, 7.0, -5.0), (25.0, 25.0, -1.5)])
def test_gz_finite_differences(orc, station):
    """d(gz)/dx = gxz, d(gz)/dy = gyz, d(gz)/dz = gzz at the station
    (fourth-order central differences of the gz closed form)."""
    box = (0.0, 10.0, 0.0, 20.0, 0.0, 15.0)
    e = 1e-2
    st = np.asarray(station, float)
    g0 = orc.prism(st, box)

    def d_dir(axis):
        def gz(off):
            s = st.copy()
            s[axis] += off
            return orc.prism(s, box)[0]

        return (-gz(2 * e) + 8 * gz(e) - 8 * gz(-e) + gz(-2 * e)) / (12 * e)

    scale = np.abs(g0[1:]).max()
    assert abs(d_dir(0) - g0[3]) <= 1e-7 * scale
    assert abs(d_dir(1) - g0[5]) <= 1e-7 * scale
    assert abs(d_dir(2) - g0[6]) <= 1e-7 * scale


@pytest.mark.parametrize("station", [(3.0, 4.0, -2.0), (-12.0, 7.0, -5.0), (25.0, 25.0, -1.5)])
def test_gx_gy_finite_differences(orc, station):
    """The horizontal first derivatives against the gradient tensor: d(gx)/dx
    = gxx, d(gx)/dy = gxy, d(gx)/dz = gxz, d(gy)/dy = gyy, d(gy)/dz = gyz
    (fourth-order central differences of the gx, gy closed forms)."""
    box = (0.0, 10.0, 0.0, 20.0, 0.0, 15.0)
    e = 1e-2
    st = np.asarray(station, float)
    g0 = orc.prism(st, box)

    def d_dir(comp, axis):
        def g(off):
            s = st.copy()
            s[axis] += off
            return orc.prism(s, box)[comp]

        return (-g(2 * e) + 8 * g(e) - 8 * g(-e) + g(-2 * e)) / (12 * e)

    scale = np.abs(g0[1:7]).max()
    GX, GY = 7, 8
    assert abs(d_dir(GX, 0) - g0[1]) <= 1e-7 * scale
    assert abs(d_dir(GX, 1) - g0[2]) <= 1e-7 * scale
    assert abs(d_dir(GX, 2) - g0[3]) <= 1e-7 * scale
    assert abs(d_dir(GY, 0) - g0[2]) <= 1e-7 * scale
    assert abs(d_dir(GY, 1) - g0[4]) <= 1e-7 * scale
    assert abs(d_dir(GY, 2) - g0[5]) <= 1e-7 * scale


def _gmesh():
    return (5, 4, 3, 10.0, 25.0, 20.0, 2.0)


def test_translation_invariance_of_G(orc):
    """G_ij depends only on the offset (l - p, m - q) and the layer n (Eq. 7):
    every layer block of G is block Toeplitz with Toeplitz blocks (Sec. 2.2.3)."""
    nx, ny, nz = 5, 4, 3
    G = orc.gmatrix(_gmesh(), ALL7)
    seen = {}
    for c in range(7):
        scale = np.abs(G[c]).max()
        for i in range(nx * ny):
            p, q = i % nx, i // nx
            for j in range(nx * ny * nz):
                l, m, n = j % nx, (j // nx) % ny, j // (nx * ny)
                key = (c, l - p, m - q, n)
                v = G[c, i, j]
                if key in seen:
                    assert abs(seen[key] - v) <= 1e-13 * scale
                else:
                    seen[key] = v
    # (2nx-1)(2ny-1) distinct values per layer and component (Eqs. 10, 22)
    assert len(seen) == 7 * (2 * nx - 1) * (2 * ny - 1) * nz


def test_reflection_parity(orc):
    """Mirroring the cell offset in x or y keeps gz, gxx, gyy, gzz, flips gxz
    under x, gyz under y and gxy under both (the symmetries of Sec. 2.2)."""
    nx, ny, nz = 5, 4, 3
    G = orc.gmatrix(_gmesh(), ALL7)
    par_x = np.array([1, 1, -1, -1, 1, 1, 1])
    par_y = np.array([1, 1, -1, 1, 1, -1, 1])
    tol = 1e-13 * np.abs(G).max(axis=(1, 2))

    def same(a, b):
        return bool(np.all(np.abs(a - b) <= tol))

    # station (2, q) sits on the mesh's x mid-line: cells l and 4 - l mirror
    for q in range(ny):
        i = 2 + nx * q
        for n in range(nz):
            for m in range(ny):
                for l in range(nx):
                    j = l + nx * m + nx * ny * n
                    jm = (nx - 1 - l) + nx * m + nx * ny * n
                    assert same(G[:, i, j], par_x * G[:, i, jm])
    # y mirror through station row q: cell m -> 2q - m when both are in range
    for p in range(nx):
        for q in range(ny):
            i = p + nx * q
            for m in range(ny):
                mm = 2 * q - m
                if not 0 <= mm < ny:
                    continue
                for n in range(nz):
                    for l in range(nx):
                        j = l + nx * m + nx * ny * n
                        jm = l + nx * mm + nx * ny * n
                        assert same(G[:, i, j], par_y * G[:, i, jm])


def test_superposition_box(orc):
    """Summing G over the cells of a uniform box (Eq. 3) gives the closed form
    of the whole box: this pins the cell and station indexing."""
    mesh = (8, 7, 5, 10.0, 12.0, 9.0, 3.0)
    box = (2, 5, 1, 6, 1, 4)
    rho = np.zeros((5, 7, 8))
    rho[1:4, 1:6, 2:5] = 250.0
    got = orc.forward(mesh, ALL7, rho)
    ref = orc.box_field(mesh, ALL7, box, 250.0).reshape(7, 7, 8)
    for c in range(7):
        scale = np.abs(ref[c]).max()
        assert np.abs(got[c] - ref[c]).max() <= 1e-11 * scale


def test_paper_cube_model_superposition(orc):
    """The Sec. 3.1 accuracy model (300 m cube, 500-800 m deep, +300 kg/m^3,
    40x40x20 mesh of 50 m cells, stations 50 m up): direct summation over the
    mesh equals the single-prism closed form of the cube."""
    mesh, rho, boxes = W.cube40()
    rng = np.random.default_rng(0)
    st = W.station_subset(mesh, 40, rng)
    got = orc.forward(mesh.tuple(), ALL7, rho, stations=st)
    l0, l1, m0, m1, n0, n1, d = boxes[0]
    ref = orc.box_field(mesh.tuple(), ALL7, (l0, l1, m0, m1, n0, n1), d, stations=st)
    for c in range(7):
        scale = np.abs(ref[c]).max()
        assert np.abs(got[c] - ref[c]).max() <= 1e-11 * scale


def test_forward_equals_explicit_G(orc):
    """The direct sum and the explicit matrix-vector product G rho agree (Eq. 4)."""
    mesh = _gmesh()
    rng = np.random.default_rng(3)
    rho = rng.uniform(-500, 500, (3, 4, 5))
    G = orc.gmatrix(mesh, ALL7)
    d = orc.forward(mesh, ALL7, rho).reshape(7, -1)
    ref = G @ rho.reshape(-1)
    assert np.allclose(d, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_adjoint_is_transpose(orc):
    """The adjoint equals the explicit transpose G^T r, summed over components."""
    mesh = _gmesh()
    rng = np.random.default_rng(4)
    comps = 0b0111011  # gz, gxx, gxz, gyy, gyz
    nc = 5
    r = rng.normal(size=(nc, 4, 5))
    G = orc.gmatrix(mesh, comps)
    ref = np.einsum("cij,ci->j", G, r.reshape(nc, -1))
    got = orc.adjoint(mesh, comps, r).reshape(-1)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    cells = np.array([0, 7, 33, 59], dtype=np.int32)
    assert np.allclose(orc.adjoint(mesh, comps, r, cells=cells), ref[cells], rtol=1e-12)


def test_station_subset_matches_full(orc):
    mesh, rho = W.small16()
    full = orc.forward(mesh.tuple(), 1 | 2, rho)
    st = np.array([0, 15, 17, 255, 130], dtype=np.int32)
    sub = orc.forward(mesh.tuple(), 1 | 2, rho, stations=st)
    assert np.array_equal(sub, full.reshape(2, -1)[:, st])


def test_invalid_arguments(orc):
    with pytest.raises(ValueError):
        orc.forward((4, 4, 1, 10.0, 10.0, 10.0, 0.0), 1, np.zeros((1, 4, 4)))  # h = 0
    with pytest.raises(ValueError):
        orc.forward((4, 4, 1, 10.0, 10.0, 10.0, 1.0), 0, np.zeros((1, 4, 4)))  # no component
