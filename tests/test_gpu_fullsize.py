"""Parity at the benchmark's full size, in the launch configuration bench.py
times: 1024 x 1024 x 100 cells (50 x 50 x 25 m, stations 10 m up), six
components.

Smooth Gaussian random field density (the bench's input, float32):
* sampled stations (the four corners, the centre and one more) against the
  CPU oracle's direct summation: FP64 spectral path <= 1e-10, FP32 <= 2e-5
  relative L2, and element-wise within the max-abs bounds below;
* the FP32 path against the FP64 path at every station: relative L2 <= 2e-5
  and max-abs within the bound.

Three-box density on the same mesh: its field is the sum of three whole-box
closed forms (superposition of Eq. 3), known exactly at every station.  Both
paths are compared element by element with it on every station of the four
edge rows and columns on each side (where a crop or wrap mistake shows) and
on every 7th station of the rest.

Max-abs bounds, per component, in mGal (gz) and Eotvos (gradients), scaled
by the component's largest value among the compared stations (of the oracle
or closed form where one is compared, of the FP64 path where FP32 is
compared with it): FP64 1e-10 x max|d_c|, FP32 2e-5 x max|d_c|.  The FP32 figure follows from the rounding model of the
FP32 path: about 46 rounding stages (row and column transforms of the
density and of the product, 2 x (11 + 11) passes at 2048 points, plus the
stored spectra and the product) of relative size 2^-24 give a normwise
relative error near 6e-8 x sqrt(46) = 4e-7 (measured 3e-7); an error spread
like noise over 1e6 stations peaks at about sqrt(2 ln 1e6) = 5.3 times its
RMS, and the fields' RMS is within a factor 10 of their peak, so the expected
peak error is about 2e-6 of the peak value: the bound leaves a factor 10,
while a localized defect (a wrong edge row, one bad kx column at 1e-4) fails
it.
"""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu

COMPS = capi.GRAV_ALL6
UNITS = np.array([1e5] + [1e9] * 5)  # m/s^2 -> mGal, 1/s^2 -> Eotvos
MAXABS64 = 1e-10
MAXABS32 = 2e-5


@pytest.fixture(scope="module")
def plans(gravlib):
    mesh = W.grf_mesh()
    p32 = Plan(mesh, COMPS, fp64=False)
    p64 = Plan(mesh, COMPS, fp64=True)
    yield mesh, p32, p64
    p32.close()
    p64.close()


@pytest.fixture(scope="module")
def grf_case(plans, orc):
    mesh, p32, p64 = plans
    _, rho = W.grf1024(device="cuda")
    rho = rho.contiguous()
    d32 = p32.forward(rho).cpu().double().numpy()
    d64 = p64.forward(rho.double()).cpu().numpy()
    st = W.station_subset(mesh, 6, np.random.default_rng(3))
    ref = orc.forward(mesh.tuple(), COMPS, rho.cpu().double().numpy(), stations=st)
    return mesh, st, ref, d32, d64


@pytest.fixture(scope="module")
def boxes_case(plans, orc):
    mesh, p32, p64 = plans
    _, rho, boxes = W.boxes1024()
    x = torch.as_tensor(rho, device="cuda")
    d32 = p32.forward(x).cpu().double().numpy().reshape(6, -1)
    d64 = p64.forward(x.double()).cpu().numpy().reshape(6, -1)
    nx, ny = mesh.nx, mesh.ny
    p = np.arange(nx * ny) % nx
    q = np.arange(nx * ny) // nx
    edge = (np.minimum(p, nx - 1 - p) < 4) | (np.minimum(q, ny - 1 - q) < 4)
    st = np.flatnonzero(edge | (np.arange(nx * ny) % 7 == 0))
    ref = sum(orc.box_field(mesh.tuple(), COMPS, b[:6], b[6], stations=st) for b in boxes)
    return st, ref, d32[:, st], d64[:, st]


def _rel(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _maxabs(got, ref):
    """Per-component largest absolute difference, in mGal / Eotvos."""
    return np.abs(got - ref).max(axis=1) * UNITS


def test_fp64_path_matches_oracle_at_sampled_stations(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    got = d64.reshape(6, -1)[:, st]
    err = _rel(got, ref)
    assert np.all(err <= 1e-10), err
    peak = np.abs(ref).max(axis=1) * UNITS  # largest oracle value among the sampled stations
    assert np.all(_maxabs(got, ref) <= MAXABS64 * peak), (_maxabs(got, ref), peak)


def test_fp32_path_matches_oracle_at_sampled_stations(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    got = d32.reshape(6, -1)[:, st]
    err = _rel(got, ref)
    assert np.all(err <= 2e-5), err
    peak = np.abs(ref).max(axis=1) * UNITS  # largest oracle value among the sampled stations
    assert np.all(_maxabs(got, ref) <= MAXABS32 * peak), (_maxabs(got, ref), peak)


def test_fp32_path_matches_fp64_path_everywhere(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    a, b = d32.reshape(6, -1), d64.reshape(6, -1)
    err = _rel(a, b)
    assert np.all(err <= 2e-5), err
    maxabs = _maxabs(a, b)
    peak = np.abs(b).max(axis=1) * UNITS
    print("FP32 vs FP64 rel L2", err, "max abs (mGal, E...)", maxabs, "peak", peak)
    assert np.all(maxabs <= MAXABS32 * peak), (maxabs, peak)


def test_box_model_every_edge_station_fp64(boxes_case):
    st, ref, d32, d64 = boxes_case
    peak = np.abs(ref).max(axis=1) * UNITS
    assert np.all(_rel(d64, ref) <= 1e-10), _rel(d64, ref)
    assert np.all(_maxabs(d64, ref) <= MAXABS64 * peak), (_maxabs(d64, ref), peak)


def test_box_model_every_edge_station_fp32(boxes_case):
    st, ref, d32, d64 = boxes_case
    peak = np.abs(ref).max(axis=1) * UNITS
    assert np.all(_rel(d32, ref) <= 2e-5), _rel(d32, ref)
    assert np.all(_maxabs(d32, ref) <= MAXABS32 * peak), (_maxabs(d32, ref), peak)


def test_stage_timing_records_every_call(gravlib):
    mesh, rho = W.small16()
    with Plan(mesh, COMPS) as plan:
        x = torch.as_tensor(rho, dtype=torch.float32).cuda()
        capi.grav_plan_set_timing(plan.handle, True)
        for _ in range(3):
            y = plan.forward(x)
        plan.adjoint(y)
        ms, nf, na = capi.grav_plan_stage_times(plan.handle)
        assert (nf, na) == (3, 1)
        assert all(v >= 0 for v in ms.values()) and ms["forward_columns"] > 0
        ms2, nf2, na2 = capi.grav_plan_stage_times(plan.handle)
        assert (nf2, na2) == (0, 0)
