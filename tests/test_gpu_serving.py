"""Serving form: continuous batching over resident plans.

Requests on meshes of different sizes arrive while others run; each result
must equal the same request computed alone (plain plan call), within the FP32
tolerance; admission respects the HBM budget; batches and graph replays
happen."""
import time

import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.batch import BatchRunner
from paper_2005_10160_gb300.pipeline import HostPipeline
from paper_2005_10160_gb300.plan import Plan
from paper_2005_10160_gb300.server import Server

pytestmark = pytest.mark.gpu

MESHES = [W.Mesh(64, 64, 16, 20.0, 20.0, 20.0, 10.0), W.Mesh(128, 128, 32, 20.0, 20.0, 20.0, 10.0),
          W.Mesh(96, 40, 8, 25.0, 20.0, 10.0, 5.0)]


def _inputs(rng, n):
    reqs = []
    for i in range(n):
        mesh = MESHES[rng.integers(len(MESHES))]
        kind = "forward" if rng.random() < 0.5 else "adjoint"
        if kind == "forward":
            data = torch.as_tensor(W.serving_density(mesh, rng), dtype=torch.float32)
        else:
            data = torch.as_tensor(rng.normal(size=(6, mesh.ny, mesh.nx)), dtype=torch.float32)
        reqs.append((kind, mesh, data))
    return reqs


def _alone(kind, mesh, data):
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        x = data.cuda()
        out = plan.forward(x) if kind == "forward" else plan.adjoint(x)
        torch.cuda.synchronize()
        return out.cpu()


def _rel(a, b):
    return float((a.double() - b.double()).norm() / b.double().norm())


def test_results_same_alone_and_in_the_mix(gravlib):
    rng = np.random.default_rng(5)
    inputs = _inputs(rng, 48)
    srv = Server(hbm_budget=8 << 30, slots=4, max_batch=4)
    try:
        reqs = []
        for kind, mesh, data in inputs:
            reqs.append(srv.submit(kind, mesh, data.cuda()))
            time.sleep(float(rng.exponential(0.002)))  # Poisson arrivals, mean 2 ms
        srv.drain()
        mixed = [r.wait(60).cpu() for r in reqs]
        stats = srv.stats()
    finally:
        srv.close()
    for (kind, mesh, data), got in zip(inputs, mixed):
        ref = _alone(kind, mesh, data)
        assert _rel(got, ref) <= 2e-5, (kind, mesh)
    assert stats["requests"] == len(inputs)
    assert np.isfinite(stats["p50_ms"]) and stats["p99_ms"] >= stats["p50_ms"]


def test_same_plan_requests_are_batched_and_replayed_from_graphs(gravlib):
    mesh = MESHES[0]
    rng = np.random.default_rng(6)
    datas = [torch.as_tensor(W.serving_density(mesh, rng), dtype=torch.float32).cuda() for _ in range(16)]
    srv = Server(hbm_budget=4 << 30, slots=2, max_batch=8)
    try:
        # hold the loop while the queue fills so that batches form
        with srv.lock:
            reqs = [srv.submit("forward", mesh, d) for d in datas]
        srv.drain()
        outs = [r.wait(60) for r in reqs]
        assert srv.batches_run < len(datas)
        # second wave: same batch sizes again, now replayed from captured graphs
        with srv.lock:
            reqs2 = [srv.submit("forward", mesh, d) for d in datas]
        srv.drain()
        outs2 = [r.wait(60) for r in reqs2]
        assert srv.graph_replays > 0
    finally:
        srv.close()
    for d, a, b in zip(datas, outs, outs2):
        ref = _alone("forward", mesh, d.cpu())
        assert _rel(a.cpu(), ref) <= 2e-5 and _rel(b.cpu(), ref) <= 2e-5


def test_admission_under_a_tight_budget(gravlib):
    """Budget for about one plan and its batch: requests on two meshes still
    all complete (plans are evicted and rebuilt), with correct results."""
    rng = np.random.default_rng(7)
    a, b = MESHES[0], MESHES[2]
    budget = int(1.5 * max(Server._plan_bytes_estimate(m.tuple(), 63, False) for m in (a, b))) + (8 << 20)
    srv = Server(hbm_budget=budget, slots=2, max_batch=2)
    try:
        items = [(m, torch.as_tensor(W.serving_density(m, rng), dtype=torch.float32)) for m in (a, b, a, b, a)]
        reqs = [srv.submit("forward", m, d.cuda()) for m, d in items]
        srv.drain()
        outs = [r.wait(60).cpu() for r in reqs]
        assert srv.used <= budget
    finally:
        srv.close()
    for (m, d), got in zip(items, outs):
        assert _rel(got, _alone("forward", m, d)) <= 2e-5


def test_request_beyond_the_budget_fails_cleanly(gravlib):
    srv = Server(hbm_budget=1 << 20, slots=1)
    try:
        mesh = MESHES[1]
        r = srv.submit("forward", mesh, torch.zeros((mesh.nz, mesh.ny, mesh.nx)).cuda())
        srv.drain()
        with pytest.raises(RuntimeError):
            r.wait(10)
    finally:
        srv.close()


@pytest.mark.parametrize("mesh", [MESHES[2], W.Mesh(6, 600, 10, 20.0, 20.0, 10.0, 5.0),
                                  W.Mesh(520, 9, 5, 20.0, 20.0, 10.0, 5.0),
                                  W.Mesh(520, 528, 3, 20.0, 20.0, 10.0, 5.0),
                                  W.Mesh(12, 300, 7, 20.0, 20.0, 10.0, 5.0)])
def test_batch_runner_matches_single_calls(gravlib, mesh):
    """grav_forward_batch / grav_adjoint_batch with a caller workspace equal
    per-request plain calls (the second mesh runs 2048-point columns, the
    third 2048-point rows, the fourth both, with the tiled adjoint, the fifth
    1024-point columns with two 512-point transforms per warp)."""
    rng = np.random.default_rng(8)
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        run = BatchRunner(plan)
        x = torch.as_tensor(rng.uniform(-300, 300, (3, mesh.nz, mesh.ny, mesh.nx)), dtype=torch.float32).cuda()
        y = run.forward(x)
        r = torch.as_tensor(rng.normal(size=(3, 6, mesh.ny, mesh.nx)), dtype=torch.float32).cuda()
        g = run.adjoint(r)
        for i in range(3):
            assert torch.equal(y[i], plan.forward(x[i].contiguous()))
            assert torch.equal(g[i], plan.adjoint(r[i].contiguous()))


def test_host_pipeline_matches_plain_calls(gravlib):
    """HostPipeline (two lanes, host-resident pinned buffers) gives for every
    request exactly what a plain forward on device buffers gives."""
    mesh = W.Mesh(520, 528, 3, 20.0, 20.0, 10.0, 5.0)
    rng = np.random.default_rng(9)
    with Plan(mesh, capi.GRAV_ALL6) as plan:
        pipe = HostPipeline(plan, lanes=2)
        rhos = [torch.as_tensor(rng.uniform(-300, 300, (mesh.nz, mesh.ny, mesh.nx)), dtype=torch.float32).pin_memory()
                for _ in range(5)]
        outs = [torch.empty((6, mesh.ny, mesh.nx), dtype=torch.float32).pin_memory() for _ in rhos]
        for rh, oh in zip(rhos, outs):
            pipe.forward(rh, oh)
        pipe.synchronize()
        for rh, oh in zip(rhos, outs):
            ref = plan.forward(rh.cuda()).cpu()
            assert torch.equal(oh, ref)
