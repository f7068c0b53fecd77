"""Host logic of the serving loop, on the CPU: which requests form a batch,
when a plan is created or an idle one evicted, when a batch waits, runs or
fails against the HBM budget, and what finishing a batch gives back.

The server is built without its constructor (which makes CUDA streams and a
worker thread); plans, launches and request sizes are fakes, and
torch.cuda.device is replaced by a null context, so no device is touched.
"""
import collections
import contextlib
import itertools
import threading

import pytest
import torch

from paper_2005_10160_gb300 import capi, server as S

MESH_A = (16, 16, 4, 10.0, 10.0, 10.0, 1.0)
MESH_B = (32, 16, 4, 10.0, 10.0, 10.0, 1.0)
MESH_C = (64, 64, 8, 10.0, 10.0, 10.0, 1.0)
MESH_A_HIGH = (16, 16, 4, 10.0, 10.0, 10.0, 50.0)  # MESH_A seen from 50 m: same shape class


class FakePlan:
    def __init__(self, mesh, comps, fp64=False):
        self.mesh, self.comps, self.fp64 = mesh, comps, fp64
        self.nbytes = HostServer.PLAN_BYTES[tuple(mesh)]
        self.closed = False

    def close(self):
        self.closed = True


class FakeSlot:
    def __init__(self, index):
        self.index, self.busy, self.batch, self.out, self.nbytes, self.graphs = index, False, [], None, 0, {}
        self.start = self.event = None


class HostServer(S.Server):
    PLAN_BYTES = {MESH_A: 1000, MESH_B: 2000, MESH_C: 5000, MESH_A_HIGH: 1000}

    def __init__(self, budget, slots=2, max_batch=8, graph_bytes_limit=1 << 20, req_bytes=(100, 50, 10)):
        self.budget, self.max_batch = budget, max_batch
        self.graph_bytes_limit, self.graph_memory = graph_bytes_limit, 1 << 30
        self.plans = collections.OrderedDict()
        self.plan_users = collections.defaultdict(int)
        self.used = self.graph_used = 0
        self.queue = collections.deque()
        self.lock = threading.Condition()
        self.slots = [FakeSlot(i) for i in range(slots)]
        self.ids = itertools.count()
        self.completed, self.batches_run, self.graph_replays = [], 0, 0
        self.max_busy_slots, self.device_intervals = 0, []
        self.building, self.cross_plan, self.plans_built = {}, True, 0
        self.device = torch.device("cpu")
        self.req_bytes = req_bytes
        self.launched = []

    @staticmethod
    def _plan_bytes_estimate(mesh, comps, fp64):
        return HostServer.PLAN_BYTES[tuple(mesh)]

    def _request_bytes(self, plan, kind):
        b_in, b_out, b_ws = self.req_bytes
        return (b_in, b_out, b_ws) if kind == "forward" else (b_out, b_in, b_ws)

    def _launch(self, slot, plan, kind, batch, use_graph, sizes):
        self.launched.append((batch[0].key, kind, [r.rid for r in batch], use_graph))
        slot.nbytes = len(batch) * sum(sizes)
        self.used += slot.nbytes
        slot.batch, slot.out, slot.busy = batch, [f"out{r.rid}" for r in batch], True
        self.batches_run += 1


@pytest.fixture(autouse=True)
def no_device(monkeypatch):
    monkeypatch.setattr(S, "Plan", FakePlan)
    monkeypatch.setattr(S.torch.cuda, "device", lambda *a, **k: contextlib.nullcontext())


def key(mesh, comps=capi.GRAV_ALL6):
    return (mesh, comps, False)


def enqueue(srv, items):
    reqs = []
    for mesh, kind in items:
        r = S.Request(kind, key(mesh), torch.zeros(1), 0.0, next(srv.ids))
        srv.queue.append(r)
        reqs.append(r)
    return reqs


def test_batch_is_the_oldest_request_and_later_ones_of_the_same_plan_and_kind():
    srv = HostServer(budget=1 << 20, max_batch=3)
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_B, "forward"), (MESH_A, "adjoint"), (MESH_A, "forward"),
                         (MESH_A, "forward"), (MESH_A, "forward")])
    assert [r.rid for r in srv._take_batch()] == [reqs[0].rid, reqs[3].rid, reqs[4].rid]  # capped at 3, in order


def test_admitted_batch_leaves_the_queue_and_holds_its_plan():
    srv = HostServer(budget=1 << 20)
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_B, "adjoint"), (MESH_A, "forward")])
    assert srv._admit(srv.slots[0])
    assert srv.launched == [(key(MESH_A), "forward", [reqs[0].rid, reqs[2].rid], True)]
    assert list(srv.queue) == [reqs[1]]
    assert srv.plan_users[key(MESH_A)] == 1
    assert srv.used == 1000 + 2 * 160  # the plan plus the batch's buffers


def test_large_requests_run_eagerly_small_ones_from_graphs():
    srv = HostServer(budget=1 << 20, graph_bytes_limit=159)  # one request is 160 bytes
    enqueue(srv, [(MESH_A, "forward")])
    assert srv._admit(srv.slots[0])
    assert srv.launched[-1][3] is False


def test_idle_plans_are_evicted_least_recently_used_first():
    srv = HostServer(budget=3500)
    for mesh in (MESH_A, MESH_B):
        srv._plan(key(mesh))
    srv._plan(key(MESH_A))  # A becomes the most recently used
    a, b = srv.plans[key(MESH_A)], srv.plans[key(MESH_B)]
    srv.slots[0].graphs[(key(MESH_B), "forward", 1)] = S._GraphEntry(None, None, None, None, 64)
    srv.graph_used = 64
    c_need = HostServer.PLAN_BYTES[MESH_C]
    srv.budget = 1000 + c_need  # room for C only once B is gone
    assert srv._plan(key(MESH_C)) is not None
    assert b.closed and not a.closed
    assert key(MESH_B) not in srv.plans and key(MESH_A) in srv.plans
    assert srv.slots[0].graphs == {} and srv.graph_used == 0  # B's captured graphs go with it
    assert srv.used == 1000 + c_need


def test_plan_in_use_is_never_evicted():
    srv = HostServer(budget=2500)
    srv._plan(key(MESH_A))
    srv.plan_users[key(MESH_A)] = 1
    assert srv._plan(key(MESH_B)) is None  # would need A's memory, but A has a batch in flight
    assert key(MESH_A) in srv.plans and not srv.plans[key(MESH_A)].closed


def test_plan_beyond_budget_waits_while_a_batch_is_in_flight_else_fails():
    srv = HostServer(budget=1500)
    reqs = enqueue(srv, [(MESH_B, "forward"), (MESH_B, "forward")])
    srv.slots[1].busy = True
    assert srv._admit(srv.slots[0]) is False and len(srv.queue) == 2  # wait: the busy batch may free memory
    srv.slots[1].busy = False
    assert srv._admit(srv.slots[0]) is True
    assert not srv.queue and all(r.done.is_set() and "HBM budget" in r.error for r in reqs)
    assert srv.launched == []


def test_request_beyond_budget_drops_graphs_and_idle_plans_first():
    srv = HostServer(budget=1000 + 2000 + 400, req_bytes=(200, 100, 50))  # A and B resident, 350 per request
    srv._plan(key(MESH_B))
    srv._plan(key(MESH_A))
    srv.slots[1].graphs[(key(MESH_B), "adjoint", 1)] = S._GraphEntry(None, None, None, None, 300)
    srv.graph_used = 300
    enqueue(srv, [(MESH_A, "forward")])
    assert srv._admit(srv.slots[0])
    assert srv.graph_used == 0 and key(MESH_B) not in srv.plans  # freed to make room
    assert srv.launched == [(key(MESH_A), "forward", [0], False)]  # eager after graphs were dropped


def test_request_that_cannot_fit_even_alone_fails_cleanly():
    srv = HostServer(budget=1200, req_bytes=(200, 100, 50))
    reqs = enqueue(srv, [(MESH_A, "forward")])
    assert srv._admit(srv.slots[0])
    assert reqs[0].done.is_set() and "beyond the HBM budget" in reqs[0].error
    assert srv.plan_users[key(MESH_A)] == 0 and not srv.queue


def test_finishing_a_batch_returns_its_memory_and_releases_the_plan():
    srv = HostServer(budget=1 << 20)
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_A, "forward")])
    srv._admit(srv.slots[0])
    srv._finish(srv.slots[0])
    assert srv.used == 1000 and srv.plan_users[key(MESH_A)] == 0 and not srv.slots[0].busy
    assert [r.result for r in reqs] == [f"out{r.rid}" for r in reqs] and all(r.done.is_set() for r in reqs)
    assert srv.completed == reqs


def test_plan_size_estimate_counts_the_compressed_spectra():
    """1024 x 1024 x 100, six components, FP32: the spectra alone are
    2 parities x 1025 kx x 100 layers x 6 components x 516 (jp) x 4 bytes."""
    spectra = 2 * 1025 * 100 * 6 * 516 * 4
    est = S.Server._plan_bytes_estimate((1024, 1024, 100, 50.0, 50.0, 25.0, 10.0), capi.GRAV_ALL6, False)
    workspaces = 2 * 1025 * 100 * 1024 * 8 + 2 * 1025 * 6 * 1024 * 8
    assert est == spectra + workspaces + 2048 * 8 + 256
    assert S.Server._plan_bytes_estimate((1024, 1024, 100, 50.0, 50.0, 25.0, 10.0), capi.GRAV_ALL6, True) > 2 * spectra


def test_device_overlap_counts_intervals_that_share_an_instant():
    """max_concurrent_on_device: the largest number of batch intervals on the
    device time line that contain one instant; touching ends do not count."""
    srv = HostServer(budget=1 << 20)
    srv.device_intervals = [(0.0, 1.0, 0), (0.5, 2.0, 1), (1.0, 3.0, 0), (1.5, 1.8, 2), (5.0, 6.0, 1)]
    assert srv.max_concurrent_on_device() == 3  # (0.5, 2), (1, 3) and (1.5, 1.8) at t = 1.6
    srv.device_intervals = [(0.0, 1.0, 0), (1.0, 2.0, 1)]
    assert srv.max_concurrent_on_device() == 1
    srv.device_intervals = []
    assert srv.max_concurrent_on_device() == 0


def test_requests_on_plans_of_one_shape_class_share_a_batch():
    """A later request of the same kind on another resident plan with the
    same mesh size, components and precision joins the batch; one on a plan
    not yet resident, or of another size, does not."""
    srv = HostServer(budget=1 << 20, max_batch=8)
    srv._plan(key(MESH_A))
    srv._plan(key(MESH_A_HIGH))
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_A_HIGH, "forward"), (MESH_B, "forward"),
                         (MESH_A_HIGH, "adjoint"), (MESH_A, "forward")])
    assert [r.rid for r in srv._take_batch()] == [reqs[0].rid, reqs[1].rid, reqs[4].rid]
    srv.cross_plan = False
    assert [r.rid for r in srv._take_batch()] == [reqs[0].rid, reqs[4].rid]
    srv.cross_plan = True
    srv.plans.pop(key(MESH_A_HIGH))
    assert [r.rid for r in srv._take_batch()] == [reqs[0].rid, reqs[4].rid]


def test_cross_plan_batch_holds_every_plan_it_uses_and_runs_eagerly():
    srv = HostServer(budget=1 << 20)
    srv._plan(key(MESH_A))
    srv._plan(key(MESH_A_HIGH))
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_A_HIGH, "forward")])
    assert srv._admit(srv.slots[0])
    assert srv.launched == [(key(MESH_A), "forward", [reqs[0].rid, reqs[1].rid], False)]
    assert srv.plan_users[key(MESH_A)] == 1 and srv.plan_users[key(MESH_A_HIGH)] == 1
    srv._finish(srv.slots[0])
    assert srv.plan_users[key(MESH_A)] == 0 and srv.plan_users[key(MESH_A_HIGH)] == 0


class AsyncHostServer(HostServer):
    """The host server with a builder: plan builds are queued, not run."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self._builder = object()
        self._build_q = __import__("queue").Queue()


def test_a_plan_being_built_does_not_hold_up_requests_on_resident_plans():
    srv = AsyncHostServer(budget=1 << 20)
    srv.plans[key(MESH_B)] = FakePlan(MESH_B, capi.GRAV_ALL6)
    srv.used = 2000
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_B, "forward")])
    assert srv._admit(srv.slots[0])
    assert key(MESH_A) in srv.building and srv._build_q.get_nowait() == key(MESH_A)
    assert srv.used == 2000 + 1000 + 160  # B, A's reservation, B's batch
    assert srv.launched == [(key(MESH_B), "forward", [reqs[1].rid], True)]
    assert list(srv.queue) == [reqs[0]]  # waits for its plan
    assert srv._admit(srv.slots[1]) is False  # still building
    srv._build_done(key(MESH_A), FakePlan(MESH_A, capi.GRAV_ALL6), None)
    assert key(MESH_A) not in srv.building and srv.plans_built == 1
    assert srv._admit(srv.slots[1])
    assert srv.launched[-1] == (key(MESH_A), "forward", [reqs[0].rid], True)


def test_a_failed_build_fails_its_requests_and_returns_the_reservation():
    srv = AsyncHostServer(budget=1 << 20)
    reqs = enqueue(srv, [(MESH_A, "forward"), (MESH_A, "adjoint")])
    assert srv._admit(srv.slots[0]) is False and srv.used == 1000
    srv._build_done(key(MESH_A), None, "GravError: no memory")
    assert srv.used == 0 and not srv.queue
    assert all(r.done.is_set() and r.error == "GravError: no memory" for r in reqs)


def test_a_plan_beyond_the_budget_waits_while_another_is_being_built():
    srv = AsyncHostServer(budget=2500)
    enqueue(srv, [(MESH_A, "forward"), (MESH_B, "forward")])
    assert srv._admit(srv.slots[0]) is False  # A building (1000), B needs 2000 more: wait
    assert list(srv.building) == [key(MESH_A)] and len(srv.queue) == 2
