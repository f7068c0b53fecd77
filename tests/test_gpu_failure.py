"""Failure detection without a GPU fault: the bounded pipeline wait gives up
and reports GRAV_ETIMEOUT, and the context stays usable afterwards."""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives(gravlib, orc):
    rc, waited = capi.grav_selftest_bounded_wait(20.0)
    assert rc == capi.GRAV_ETIMEOUT, capi.grav_last_error()
    assert 20.0 <= waited < 2000.0
    # the device still works: a forward after the timed-out wait is correct
    mesh, rho = W.small16()
    with Plan(mesh, capi.GRAV_GZ, fp64=True) as plan:
        out = plan.forward(torch.as_tensor(rho, dtype=torch.float64).cuda())
        capi.grav_plan_check(plan.handle)  # no pipeline wait ran out
        got = out.cpu().numpy()
    ref = orc.forward(mesh.tuple(), capi.GRAV_GZ, rho)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_selftest_rejects_bad_limit(gravlib):
    rc, _ = capi.grav_selftest_bounded_wait(-1.0)
    assert rc == capi.GRAV_EINVAL
