"""The forward entry point that allocates nothing.

grav_forward_static_scratch serves callers that cannot call cudaMalloc once
running (device memory reserved by another framework's allocator, or a
serving loop that must not risk cudaMalloc's device synchronisation): it
runs the same forward as grav_forward with its scratch taken from the
library's static device array.  Called through the C ABI here, twice in a
row with different densities, and compared with grav_forward on the same
plan.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64,tol", [(False, 2e-5), (True, 1e-10)])
@pytest.mark.parametrize("mesh", [(16, 16, 4, 10.0, 10.0, 10.0, 1.0), (37, 29, 5, 20.0, 20.0, 15.0, 4.0),
                                  (128, 128, 32, 20.0, 20.0, 20.0, 10.0)])
def test_static_scratch_forward_matches_grav_forward(gravlib, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    dt = torch.float64 if fp64 else torch.float32
    rng = np.random.default_rng(nx + ny + nz)
    with Plan(mesh, capi.GRAV_ALL6, fp64=fp64) as plan:
        stream = torch.cuda.current_stream()
        for call in range(2):
            rho = torch.as_tensor(rng.uniform(-500, 500, (nz, ny, nx)), dtype=dt).cuda()
            ref = plan.forward(rho)
            out = torch.full_like(ref, float("nan"))
            rc = gravlib.grav_forward_static_scratch(plan.handle, rho.data_ptr(), out.data_ptr(),
                                                     stream.cuda_stream)
            assert rc == capi.GRAV_OK, capi.grav_last_error()
            torch.cuda.synchronize()
            err = (torch.linalg.vector_norm((out - ref).reshape(6, -1), dim=1)
                   / torch.linalg.vector_norm(ref.reshape(6, -1), dim=1))
            assert torch.all(err <= tol), (call, err)


def test_static_scratch_rejects_plans_too_large(gravlib):
    mesh = (256, 256, 32, 25.0, 25.0, 20.0, 5.0)
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        rho = torch.zeros((32, 256, 256), dtype=torch.float32, device="cuda")
        out = torch.empty((6, 256, 256), dtype=torch.float32, device="cuda")
        rc = gravlib.grav_forward_static_scratch(plan.handle, rho.data_ptr(), out.data_ptr(), None)
        assert rc == capi.GRAV_EINVAL
        assert "static area holds" in capi.grav_last_error()
