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


def _oracle_sample(orc, kind, mesh, data, got, rng):
    """Relative L2 error of a served result against the CPU oracle's direct
    summation at 8 sampled stations (forward, per component) or cells
    (adjoint)."""
    if kind == "forward":
        st = W.station_subset(mesh, 8, rng)
        want = orc.forward(mesh.tuple(), capi.GRAV_ALL6, data.double().numpy(), stations=st)
        have = got.reshape(6, -1)[:, st].double().numpy()
        return np.linalg.norm(have - want, axis=1) / np.linalg.norm(want, axis=1)
    cells = rng.choice(mesh.nx * mesh.ny * mesh.nz, 8, replace=False)
    want = orc.adjoint(mesh.tuple(), capi.GRAV_ALL6, data.double().numpy(), cells=cells)
    have = got.reshape(-1)[cells].double().numpy()
    return np.array([np.linalg.norm(have - want) / np.linalg.norm(want)])


def test_results_same_alone_and_in_the_mix(gravlib, orc):
    """Requests arrive in bursts of 8 (so that several batches are in flight
    on the slots' streams at once) on three meshes, forward and adjoint
    mixed.  Every served result equals the same request run alone (<= 2e-5)
    and the CPU oracle at sampled stations or cells (FP32 bar, 2e-5), and
    the device time line shows batches overlapping."""
    rng = np.random.default_rng(5)
    inputs = _inputs(rng, 48)
    srv = Server(hbm_budget=8 << 30, slots=4, max_batch=4)
    try:
        reqs = []
        for b in range(0, len(inputs), 8):
            # a burst of 8 enters the queue at once, so that one sweep of the
            # loop admits a batch into every free slot
            with srv.lock:
                reqs += [srv.submit(kind, mesh, data.cuda()) for kind, mesh, data in inputs[b:b + 8]]
            time.sleep(float(rng.exponential(0.004)))  # Poisson gaps between bursts
        srv.drain()
        mixed = [r.wait(60).cpu() for r in reqs]
        stats = srv.stats()
    finally:
        srv.close()
    srng = np.random.default_rng(55)
    for (kind, mesh, data), got in zip(inputs, mixed):
        ref = _alone(kind, mesh, data)
        assert _rel(got, ref) <= 2e-5, (kind, mesh)
        err = _oracle_sample(orc, kind, mesh, data, got, srng)
        assert np.all(err <= 2e-5), (kind, mesh, err)
    assert stats["requests"] == len(inputs)
    assert np.isfinite(stats["p50_ms"]) and stats["p99_ms"] >= stats["p50_ms"]
    assert stats["max_busy_slots"] >= 2, stats


def test_batches_on_different_slots_overlap_on_the_device(gravlib):
    """Four batches (forward and adjoint on two meshes, four requests each)
    admitted in one sweep run on four slot streams; their intervals on the
    device time line (events before and after each batch) overlap, and each
    result equals the request run alone."""
    meshes = [W.Mesh(256, 256, 32, 20.0, 20.0, 20.0, 10.0), W.Mesh(200, 180, 24, 20.0, 20.0, 20.0, 10.0)]
    rng = np.random.default_rng(12)
    groups = []
    for m in meshes:
        groups.append([("forward", m, torch.as_tensor(W.serving_density(m, rng), dtype=torch.float32))
                       for _ in range(4)])
        groups.append([("adjoint", m, torch.as_tensor(rng.normal(size=(6, m.ny, m.nx)), dtype=torch.float32))
                       for _ in range(4)])
    srv = Server(hbm_budget=16 << 30, slots=4, max_batch=4, graph_bytes_limit=0)
    try:
        for g in groups:  # build the plans first
            srv.submit(g[0][0], g[0][1], g[0][2].cuda())
        srv.drain()
        srv.device_intervals.clear()
        with srv.lock:
            reqs = [srv.submit(kind, m, d.cuda()) for g in groups for kind, m, d in g]
        srv.drain()
        outs = [r.wait(60).cpu() for r in reqs]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["max_busy_slots"] == 4, stats
    assert stats["max_concurrent_on_device"] >= 2, (stats, srv.device_intervals)
    items = [it for g in groups for it in g]
    for (kind, m, d), got in zip(items, outs):
        assert _rel(got, _alone(kind, m, d)) <= 2e-5, (kind, m)


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


@pytest.mark.parametrize("mesh,comps,fp64", [
    (W.Mesh(96, 40, 8, 25.0, 20.0, 10.0, 5.0), capi.GRAV_ALL6, False),      # generic column kernels
    (W.Mesh(6, 600, 10, 20.0, 20.0, 10.0, 5.0), capi.GRAV_ALL6, False),     # 2048-point warp columns
    (W.Mesh(12, 300, 7, 20.0, 20.0, 10.0, 5.0), capi.GRAV_ALL6, False),     # 1024-point columns, 2 per warp
    (W.Mesh(12, 300, 7, 20.0, 20.0, 10.0, 5.0), 0x1BF, False),              # 8 components: the fallback kernel
    (W.Mesh(520, 528, 3, 20.0, 20.0, 10.0, 5.0), capi.GRAV_ALL6, False),    # 2048-point rows, tiled adjoint
    (W.Mesh(37, 29, 5, 20.0, 20.0, 15.0, 4.0), capi.GRAV_ALL6, True),       # FP64
])
def test_batch_across_plans_matches_single_calls(gravlib, mesh, comps, fp64):
    """grav_forward_batch_plans / grav_adjoint_batch_plans over three plans of
    one mesh size (station heights 5, 20 and 60 m, the last with larger
    cells): every request equals, bit for bit, the plain call on its own
    plan."""
    rng = np.random.default_rng(21)
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    meshes = [mesh, W.Mesh(nx, ny, nz, mesh.dx, mesh.dy, mesh.dz, 20.0),
              W.Mesh(nx, ny, nz, 2 * mesh.dx, mesh.dy, 1.5 * mesh.dz, 60.0)]
    plans = [Plan(m, comps, fp64=fp64) for m in meshes]
    dt = torch.float64 if fp64 else torch.float32
    try:
        B = len(plans)
        nc = plans[0].ncomp
        ws = torch.empty(B * capi.grav_workspace_bytes(plans[0].handle) + 256, dtype=torch.uint8, device="cuda")
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        x = torch.as_tensor(rng.uniform(-300, 300, (B, nz, ny, nx)), dtype=dt).cuda()
        y = torch.empty((B, nc, ny, nx), dtype=dt, device="cuda")
        capi.grav_forward_batch_plans([p.handle for p in plans], x.data_ptr(), y.data_ptr(), ws_ptr,
                                      torch.cuda.current_stream().cuda_stream)
        r = torch.as_tensor(rng.normal(size=(B, nc, ny, nx)), dtype=dt).cuda()
        g = torch.empty((B, nz, ny, nx), dtype=dt, device="cuda")
        capi.grav_adjoint_batch_plans([p.handle for p in plans], r.data_ptr(), g.data_ptr(), ws_ptr,
                                      torch.cuda.current_stream().cuda_stream)
        for i, p in enumerate(plans):
            assert torch.equal(y[i], p.forward(x[i].contiguous())), i
            assert torch.equal(g[i], p.adjoint(r[i].contiguous())), i
        # plans that differ in more than their spectra are refused
        with Plan(W.Mesh(nx, ny, nz + 1, mesh.dx, mesh.dy, mesh.dz, 5.0), comps, fp64=fp64) as other:
            with pytest.raises(capi.GravError):
                capi.grav_forward_batch_plans([plans[0].handle, other.handle], x.data_ptr(), y.data_ptr(), ws_ptr,
                                              torch.cuda.current_stream().cuda_stream)
    finally:
        for p in plans:
            p.close()


def test_server_batches_requests_across_plans_of_one_size(gravlib, orc):
    """Forward and adjoint requests on one 128 x 128 x 32 model seen from two
    heights (10 m and 50 m): queued together they run as cross-plan batches;
    each result equals the request run alone and matches the CPU oracle at
    sampled stations or cells."""
    low = W.Mesh(128, 128, 32, 20.0, 20.0, 20.0, 10.0)
    high = W.Mesh(128, 128, 32, 20.0, 20.0, 20.0, 50.0)
    rng = np.random.default_rng(31)
    items = []
    for i in range(8):
        m = low if i % 2 == 0 else high
        items.append(("forward", m, torch.as_tensor(W.serving_density(m, rng), dtype=torch.float32)))
        items.append(("adjoint", m, torch.as_tensor(rng.normal(size=(6, m.ny, m.nx)), dtype=torch.float32)))
    srv = Server(hbm_budget=8 << 30, slots=2, max_batch=8)
    try:
        for m in (low, high):  # plans first
            srv.submit("forward", m, torch.zeros((m.nz, m.ny, m.nx))).wait(120)
        with srv.lock:
            reqs = [srv.submit(kind, m, d.cuda()) for kind, m, d in items]
        srv.drain()
        outs = [r.wait(60).cpu() for r in reqs]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["cross_plan_batches"] >= 2, stats
    srng = np.random.default_rng(32)
    for (kind, m, d), got in zip(items, outs):
        assert torch.equal(got, _alone(kind, m, d)), (kind, m)
        err = _oracle_sample(orc, kind, m, d, got, srng)
        assert np.all(err <= 2e-5), (kind, m, err)
