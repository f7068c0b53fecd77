"""The forward entry point that allocates nothing.

grav_forward_static_scratch serves callers that cannot call cudaMalloc once
running: a process whose device memory is all reserved by another
framework's caching allocator, or a serving loop that must not risk
cudaMalloc's device synchronisation.  It runs the same kernels as
grav_forward, with its scratch taken from the library's static device array
instead of the plan's workspaces.

Called through the C ABI here, twice in a row with different densities:
each result must equal grav_forward's on the same plan bit for bit (same
kernels, same inputs), match the CPU oracle at sampled stations (FP32
<= 2e-5, FP64 <= 1e-10 relative L2 per component), and the calls after the
first must leave the device's free memory and torch's reserved memory
unchanged.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu

MESHES = [(16, 16, 4, 10.0, 10.0, 10.0, 1.0), (37, 29, 5, 20.0, 20.0, 15.0, 4.0),
          (128, 128, 32, 20.0, 20.0, 20.0, 10.0)]


def _static_forward(gravlib, plan, rho, out, stream):
    rc = gravlib.grav_forward_static_scratch(plan.handle, rho.data_ptr(), out.data_ptr(), stream.cuda_stream)
    assert rc == capi.GRAV_OK, capi.grav_last_error()


@pytest.mark.parametrize("fp64,tol", [(False, 2e-5), (True, 1e-10)])
@pytest.mark.parametrize("mesh", MESHES)
def test_static_scratch_forward_matches_grav_forward(gravlib, orc, mesh, fp64, tol):
    nx, ny, nz = mesh[:3]
    dt = torch.float64 if fp64 else torch.float32
    rng = np.random.default_rng(nx + ny + nz)
    st = W.station_subset(W.Mesh(*mesh), 8, np.random.default_rng(1))
    with Plan(mesh, capi.GRAV_ALL6, fp64=fp64) as plan:
        stream = torch.cuda.current_stream()
        for call in range(2):
            rho = torch.as_tensor(rng.uniform(-500, 500, (nz, ny, nx)), dtype=dt).cuda()
            ref = plan.forward(rho)
            out = torch.full_like(ref, float("nan"))
            _static_forward(gravlib, plan, rho, out, stream)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), call
            want = orc.forward(mesh, capi.GRAV_ALL6, rho.cpu().double().numpy(), stations=st)
            got = out.reshape(6, -1)[:, st].cpu().double().numpy()
            err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
            assert np.all(err <= tol), (call, err)


def test_static_scratch_allocates_nothing(gravlib):
    """After the first call (which looks up the static array's address),
    further calls change neither the device's free memory nor the memory
    torch's allocator holds."""
    mesh = MESHES[2]
    nx, ny, nz = mesh[:3]
    rng = np.random.default_rng(11)
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        stream = torch.cuda.current_stream()
        rhos = [torch.as_tensor(rng.uniform(-500, 500, (nz, ny, nx)), dtype=torch.float32).cuda() for _ in range(3)]
        outs = [torch.empty((6, ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
        _static_forward(gravlib, plan, rhos[0], outs[0], stream)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        for rho, out in zip(rhos[1:], outs[1:]):
            _static_forward(gravlib, plan, rho, out, stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_reserved() == reserved0
        for rho, out in zip(rhos[1:], outs[1:]):
            assert torch.equal(out, plan.forward(rho))


def test_static_scratch_rejects_plans_too_large(gravlib):
    mesh = (256, 256, 32, 25.0, 25.0, 20.0, 5.0)
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        rho = torch.zeros((32, 256, 256), dtype=torch.float32, device="cuda")
        out = torch.empty((6, 256, 256), dtype=torch.float32, device="cuda")
        rc = gravlib.grav_forward_static_scratch(plan.handle, rho.data_ptr(), out.data_ptr(), None)
        assert rc == capi.GRAV_EINVAL
        assert "static area holds" in capi.grav_last_error()
