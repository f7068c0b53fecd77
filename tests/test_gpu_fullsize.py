"""Parity at the benchmark's full size, in the launch configuration bench.py
times: 1024 x 1024 x 100 cells (50 x 50 x 25 m, stations 10 m up), smooth
Gaussian random field density in float32, six components.

* sampled stations (the four corners, the centre and one more) against the
  CPU oracle's direct summation: FP64 spectral path <= 1e-10, FP32 <= 2e-5;
* the FP32 path against the FP64 path over the whole field: <= 2e-5.
"""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu

COMPS = capi.GRAV_ALL6


@pytest.fixture(scope="module")
def grf_case(gravlib, orc):
    mesh, rho = W.grf1024(device="cuda")
    rho = rho.contiguous()
    with Plan(mesh, COMPS, fp64=False) as p32:
        d32 = p32.forward(rho).cpu().double().numpy()
    with Plan(mesh, COMPS, fp64=True) as p64:
        d64 = p64.forward(rho.double()).cpu().numpy()
    st = W.station_subset(mesh, 6, np.random.default_rng(3))
    ref = orc.forward(mesh.tuple(), COMPS, rho.cpu().double().numpy(), stations=st)
    return mesh, st, ref, d32, d64


def _rel(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def test_fp64_path_matches_oracle_at_sampled_stations(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    err = _rel(d64.reshape(6, -1)[:, st], ref)
    assert np.all(err <= 1e-10), err


def test_fp32_path_matches_oracle_at_sampled_stations(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    err = _rel(d32.reshape(6, -1)[:, st], ref)
    assert np.all(err <= 2e-5), err


def test_fp32_path_matches_fp64_path_everywhere(grf_case):
    mesh, st, ref, d32, d64 = grf_case
    err = _rel(d32.reshape(6, -1), d64.reshape(6, -1))
    assert np.all(err <= 2e-5), err
    # max-abs in mGal (gz) and Eotvos (gradients), for the record
    scale = np.array([1e5] + [1e9] * 5)
    maxabs = np.abs(d32 - d64).reshape(6, -1).max(axis=1) * scale
    print("FP32 vs FP64 rel L2", err, "max abs (mGal, E...)", maxabs)


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
