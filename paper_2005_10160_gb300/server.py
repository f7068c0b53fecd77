"""Continuous-batching request loop over resident plans.

Forward and adjoint requests on meshes of different sizes arrive at any
time.  The loop keeps each mesh's plan (its kernel spectra, Eq. 22) resident
on the device, admits queued requests into execution slots as slots and
device memory free up, groups queued requests of the same kind into one
batched call (one launch per stage for the whole batch), runs each slot on
its own CUDA stream so that work of different slots overlaps on the GPU, and
records per-request latency from submission to the completion of its batch
on the device.

A batch is the oldest admissible request plus later ones of the same kind on
the same plan, or on another resident plan of the same mesh size,
components and precision (plans that differ only in cell size or station
height, e.g. one model seen from several survey heights): those share the
padded FFT sizes and run in one launch per stage with a per-request table of
kernel spectra (grav_forward_batch_plans).

Plans are built by a builder thread, off the admission lock: a request whose
plan is not resident waits in the queue while later requests on resident
plans keep being admitted.  Each slot has a waiter thread that blocks on its
batch's completion event and hands the results back, so completion costs no
polling.

Admission is by an HBM budget: resident plans and plans being built, plus,
for every batch in flight, its input, output and workspace buffers.  A plan
that is not in use may be evicted (least recently used) to admit another.
Small single-plan batches are replayed from CUDA graphs captured per (slot,
plan, kind, batch size).

All arithmetic happens in libgravfft.so through the C ABI.
"""
from __future__ import annotations

import collections
import itertools
import queue as queue_mod
import sys
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi
from .plan import Plan


@dataclass(eq=False)
class Request:
    kind: str                 # "forward" or "adjoint"
    key: tuple                # (mesh tuple, components, fp64)
    data: torch.Tensor        # device input: rho [nz][ny][nx] or r [ncomp][ny][nx]
    t_submit: float
    rid: int
    ready: torch.cuda.Event | None = None  # input ready on the submitting stream
    result: torch.Tensor | None = None
    t_done: float | None = None
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return (self.t_done - self.t_submit) if self.t_done is not None else float("nan")

    def wait(self, timeout=None) -> torch.Tensor:
        if not self.done.wait(timeout):
            raise TimeoutError(f"request {self.rid} not finished")
        if self.error:
            raise RuntimeError(self.error)
        return self.result


def shape_class(key) -> tuple:
    """What plans must share for their requests to run in one batched call:
    mesh sizes, components and precision (not cell sizes or height)."""
    mesh, comps, fp64 = key
    return (tuple(mesh[:3]), comps, fp64)


class _GraphEntry:
    def __init__(self, graph, inp, out, ws, nbytes):
        self.graph, self.inp, self.out, self.ws, self.nbytes = graph, inp, out, ws, nbytes


class _Slot:
    def __init__(self, device, index):
        self.index = index
        self.stream = torch.cuda.Stream(device=device)
        self.busy = False
        self.event = None
        self.start = None  # timing event recorded on the slot's stream before its batch
        self.batch: list[Request] = []
        self.buffers = ()
        self.nbytes = 0
        self.out = None
        self.graphs: dict = {}


class Server:
    """hbm_budget: bytes the server may hold on the device (plans + batches in
    flight + captured graphs).  slots: concurrent batches.  max_batch: most
    requests per batched call (at most 16 when they span several plans).
    graph_bytes_limit: per-request size (input + output + workspace) below
    which single-plan batches are replayed from CUDA graphs.  cross_plan:
    batch requests on different plans of one shape class.  switch_interval:
    the interpreter's thread switch interval while the server runs (seconds;
    None leaves it alone): a waiter thread woken by a finished batch needs the
    interpreter lock, and at the default 5 ms a busy thread can keep it that
    long, which shows in the latency tail."""

    MAX_PLANS_PER_BATCH = 16

    def __init__(self, hbm_budget: int, slots: int = 4, max_batch: int = 8, device=None,
                 graph_bytes_limit: int = 64 << 20, graph_memory: int = 2 << 30, cross_plan: bool = True,
                 switch_interval: float | None = 2e-4):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.graph_bytes_limit = int(graph_bytes_limit)
        self.graph_memory = int(graph_memory)
        self.cross_plan = bool(cross_plan)
        self.plans: "collections.OrderedDict[tuple, Plan]" = collections.OrderedDict()
        self.plan_users: dict[tuple, int] = collections.defaultdict(int)
        self.building: dict[tuple, int] = {}  # key -> bytes reserved while its plan is built
        self.used = 0
        self.graph_used = 0
        self.queue: collections.deque[Request] = collections.deque()
        self.lock = threading.Condition()
        self.slots = [_Slot(self.device, i) for i in range(slots)]
        self.ids = itertools.count()
        self.completed: list[Request] = []
        self.batches_run = 0
        self.graph_replays = 0
        self.cross_plan_batches = 0
        self.plans_built = 0
        self.max_busy_slots = 0
        # device time line: every batch's [start, end] in ms after the
        # reference event, from events on the slot streams (one GPU clock)
        self.device_intervals: list[tuple[float, float, int]] = []
        self._ref_event = torch.cuda.Event(enable_timing=True)
        with torch.cuda.device(self.device):
            self._ref_event.record(torch.cuda.current_stream(self.device))
        self._stop = False
        self._old_switch = None
        if switch_interval is not None:
            self._old_switch = sys.getswitchinterval()
            sys.setswitchinterval(min(self._old_switch, float(switch_interval)))
        self._build_q: queue_mod.Queue = queue_mod.Queue()
        self._builder = threading.Thread(target=self._build_loop, name="grav-builder", daemon=True)
        self._builder.start()
        self._waiters = [threading.Thread(target=self._wait_loop, args=(s,), name=f"grav-wait-{s.index}",
                                          daemon=True) for s in self.slots]
        for t in self._waiters:
            t.start()
        self._thread = threading.Thread(target=self._loop, name="grav-server", daemon=True)
        self._thread.start()

    # ---------------------------------------------------------------- public
    def submit(self, kind: str, mesh, data: torch.Tensor, components: int = capi.GRAV_ALL6,
               fp64: bool = False) -> Request:
        if kind not in ("forward", "adjoint"):
            raise ValueError("kind must be 'forward' or 'adjoint'")
        if hasattr(mesh, "tuple"):
            mesh = mesh.tuple()
        key = (tuple(mesh), int(components), bool(fp64))
        dt = torch.float64 if fp64 else torch.float32
        data = data.to(device=self.device, dtype=dt).contiguous()
        req = Request(kind, key, data, time.perf_counter(), next(self.ids))
        req.ready = torch.cuda.Event()
        req.ready.record(torch.cuda.current_stream(self.device))
        with self.lock:
            self.queue.append(req)
            self.lock.notify_all()
        return req

    def drain(self, timeout: float = 300.0):
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.lock:
            while self.queue or self.building or any(s.busy for s in self.slots):
                if time.perf_counter() - t0 > timeout:
                    raise TimeoutError("server did not drain")
                self.lock.wait(0.01)

    def close(self):
        self.drain()
        with self.lock:
            self._stop = True
            self.lock.notify_all()
        self._build_q.put(None)
        self._thread.join()
        for t in self._waiters:
            t.join()
        self._builder.join()
        for slot in self.slots:
            slot.graphs.clear()
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        if self._old_switch is not None:
            sys.setswitchinterval(self._old_switch)
            self._old_switch = None

    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.completed if r.error is None])
        if lat.size == 0:
            return {"requests": 0}
        span = max(r.t_done for r in self.completed) - min(r.t_submit for r in self.completed)
        return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "req_per_s": float(lat.size / span) if span > 0 else None, "batches": self.batches_run,
                "graph_replays": self.graph_replays, "cross_plan_batches": self.cross_plan_batches,
                "plans_built": self.plans_built, "max_busy_slots": self.max_busy_slots,
                "max_concurrent_on_device": self.max_concurrent_on_device()}

    def max_concurrent_on_device(self) -> int:
        """Largest number of batches whose device intervals (from the event
        before a batch's first kernel to the event after its last, on its
        slot's stream) overlap at one instant."""
        marks = []
        for t0, t1, _ in self.device_intervals:
            marks.append((t0, 1))
            marks.append((t1, -1))
        marks.sort(key=lambda m: (m[0], m[1]))  # an end before a start at the same instant
        best = cur = 0
        for _, d in marks:
            cur += d
            best = max(best, cur)
        return best

    # -------------------------------------------------------------- internals
    def _make_room(self, need: int, keep=()) -> bool:
        """Evict idle plans (least recently used first, with their captured
        graphs) until `need` more bytes fit the budget; False if they cannot."""
        while self.used + need > self.budget:
            idle = [k for k in self.plans if self.plan_users[k] == 0 and k not in keep]
            if not idle:
                return False
            victim = idle[0]
            p = self.plans.pop(victim)
            self.used -= p.nbytes
            for slot in self.slots:
                for gk in [g for g in slot.graphs if g[0] == victim]:
                    self.graph_used -= slot.graphs.pop(gk).nbytes
            p.close()
        return True

    def _plan(self, key) -> Plan | None:
        """Resident plan for key, created now (evicting idle plans) if needed;
        None while the budget cannot hold it yet."""
        if key in self.plans:
            self.plans.move_to_end(key)
            return self.plans[key]
        mesh, comps, fp64 = key
        if not self._make_room(self._plan_bytes_estimate(mesh, comps, fp64)):
            return None
        with torch.cuda.device(self.device):
            p = Plan(mesh, comps, fp64=fp64)
        self.plans[key] = p
        self.used += p.nbytes
        self.plans_built = getattr(self, "plans_built", 0) + 1
        return p

    def _start_plan(self, key) -> str | None:
        """"resident" when key's plan is on the device, "building" when the
        builder thread has it, None when the budget cannot hold it yet.
        Without a builder thread the plan is made here."""
        if key in self.plans:
            self.plans.move_to_end(key)
            return "resident"
        if key in self.building:
            return "building"
        if getattr(self, "_builder", None) is None:
            return "resident" if self._plan(key) is not None else None
        need = self._plan_bytes_estimate(*key)
        if not self._make_room(need):
            return None
        self.building[key] = need
        self.used += need
        self._build_q.put(key)
        return "building"

    def _fail_key(self, key, message: str):
        for r in [r for r in self.queue if r.key == key]:
            self.queue.remove(r)
            r.error = message
            r.t_done = time.perf_counter()
            r.done.set()

    @staticmethod
    def _plan_bytes_estimate(mesh, comps, fp64) -> int:
        nx, ny, nz = mesh[:3]
        px = 4
        while px < 2 * nx - 1:
            px *= 2
        py = 4
        while py < 2 * ny - 1:
            py *= 2
        nc = bin(comps & capi.GRAV_COMP_BITS).count("1")
        real = 8 if fp64 else 4
        kx = px // 2 + 1
        ny_pad = (ny + 3) // 4 * 4
        jp = (py // 4 + 1 + 3) // 4 * 4
        return (2 * kx * nz * nc * jp * real + 2 * kx * nz * ny_pad * 2 * real + 2 * kx * nc * ny_pad * 2 * real
                + max(px, py) * 2 * real + 256)

    def _request_bytes(self, plan: Plan, kind: str) -> tuple[int, int, int]:
        nx, ny, nz = plan.mesh[:3]
        real = 8 if plan.fp64 else 4
        rho = nz * ny * nx * real
        dat = plan.ncomp * ny * nx * real
        ws = capi.grav_workspace_bytes(plan.handle)
        return (rho, dat, ws) if kind == "forward" else (dat, rho, ws)

    def _take_batch(self, head=None):
        """`head` (default: the oldest request) plus later queued ones of the
        same kind on the same plan, or on another resident plan of the same
        shape class, capped at max_batch."""
        head = self.queue[0] if head is None else head
        batch = [head]
        cls = shape_class(head.key)
        cap = self.max_batch
        started = False
        for r in self.queue:
            if r is head:
                started = True
                continue
            if not started:
                continue
            if len(batch) >= cap:
                break
            if r.kind != head.kind:
                continue
            if r.key == head.key:
                batch.append(r)
            elif getattr(self, "cross_plan", False) and shape_class(r.key) == cls and r.key in self.plans:
                batch.append(r)
                cap = min(cap, self.MAX_PLANS_PER_BATCH)
        return batch[:cap]

    def _admit(self, slot: _Slot) -> bool:
        """Launch one batch into `slot`, or fail requests that can never fit.
        False when nothing can be admitted now."""
        head = None
        for r in list(self.queue):
            state = self._start_plan(r.key)
            if state == "resident":
                head = r
                break
            if state == "building":
                continue  # later requests on resident plans go first
            # the plan does not fit the budget now
            if any(s.busy for s in self.slots) or self.building:
                return False  # a batch in flight or a finished build may change that
            need = self._plan_bytes_estimate(*r.key)
            self._fail_key(r.key, f"the plan needs {need} bytes beyond the HBM budget of {self.budget}")
            return True
        if head is None:
            return False
        batch = self._take_batch(head)
        kind = head.kind
        keys = list(dict.fromkeys(r.key for r in batch))
        for k in keys:
            self.plans.move_to_end(k)
        plan = self.plans[head.key]
        b_in, b_out, b_ws = self._request_bytes(plan, kind)
        per_req = b_in + b_out + b_ws
        use_graph = per_req <= self.graph_bytes_limit and len(keys) == 1
        gkey = (head.key, kind, len(batch))
        # a graph replay needs only the cloned output; an eager batch its buffers
        need = len(batch) * (b_out if (use_graph and gkey in slot.graphs) else per_req)
        if self.used + self.graph_used + need > self.budget:
            if any(s.busy for s in self.slots) or self.building:
                return False  # wait for a batch in flight or a build to settle
            # nothing in flight will free memory: drop captured graphs and idle
            # plans, then fail the batch if it still does not fit
            for s in self.slots:
                for g in list(s.graphs):
                    self.graph_used -= s.graphs.pop(g).nbytes
            for k in [k for k in self.plans if k not in keys and self.plan_users[k] == 0]:
                self.used -= self.plans[k].nbytes
                self.plans.pop(k).close()
            if self.used + len(batch) * per_req > self.budget:
                for r in batch:
                    self.queue.remove(r)
                    r.error = f"request needs {per_req} bytes beyond the HBM budget of {self.budget}"
                    r.t_done = time.perf_counter()
                    r.done.set()
                return True
            use_graph = False
        for r in batch:
            self.queue.remove(r)
        for k in keys:
            self.plan_users[k] += 1
        self._launch(slot, plan, kind, batch, use_graph, (b_in, b_out, b_ws))
        return True

    def _launch(self, slot: _Slot, plan: Plan, kind: str, batch: list[Request], use_graph: bool, sizes):
        b_in, b_out, b_ws = sizes
        B = len(batch)
        nx, ny, nz = plan.mesh[:3]
        out_shape = (nz, ny, nx) if kind == "adjoint" else (plan.ncomp, ny, nx)
        in_shape = tuple(batch[0].data.shape)
        dt = plan.dtype
        plans = [self.plans[r.key] for r in batch]
        cross = any(p is not plan for p in plans)
        call = capi.grav_forward_batch if kind == "forward" else capi.grav_adjoint_batch
        gkey = (batch[0].key, kind, B)
        with torch.cuda.device(self.device), torch.cuda.stream(slot.stream):
            for r in batch:  # inputs were produced on the submitting thread's stream
                slot.stream.wait_event(r.ready)
                r.data.record_stream(slot.stream)
            start = torch.cuda.Event(enable_timing=True)
            start.record(slot.stream)
            if use_graph and not cross:
                entry = slot.graphs.get(gkey)
                if entry is None and self.graph_used + B * (b_in + b_out + b_ws) <= self.graph_memory:
                    entry = self._capture(slot, plan, call, B, in_shape, out_shape, dt, b_ws)
                    slot.graphs[gkey] = entry
                if entry is not None:
                    torch.stack([r.data for r in batch], out=entry.inp)
                    entry.graph.replay()
                    out = entry.out.clone()
                    self.graph_replays += 1
                    slot.nbytes = out.numel() * out.element_size()
                else:
                    use_graph = False
            if not use_graph or cross:
                inp = torch.stack([r.data for r in batch])
                out = torch.empty((B,) + out_shape, dtype=dt, device=self.device)
                ws = torch.empty(B * b_ws + 256, dtype=torch.uint8, device=self.device)
                ws_ptr = (ws.data_ptr() + 255) // 256 * 256
                if cross:
                    multi = capi.grav_forward_batch_plans if kind == "forward" else capi.grav_adjoint_batch_plans
                    multi([p.handle for p in plans], inp.data_ptr(), out.data_ptr(), ws_ptr, slot.stream.cuda_stream)
                    self.cross_plan_batches += 1
                else:
                    call(plan.handle, B, inp.data_ptr(), out.data_ptr(), ws_ptr, slot.stream.cuda_stream)
                slot.buffers = (inp, ws)
                slot.nbytes = B * (b_in + b_out + b_ws)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(slot.stream)
        self.used += slot.nbytes
        slot.out = out
        slot.event = ev
        slot.start = start
        slot.batch = batch
        slot.busy = True
        self.batches_run += 1
        self.max_busy_slots = max(self.max_busy_slots, sum(s.busy for s in self.slots))

    def _capture(self, slot, plan, call, B, in_shape, out_shape, dt, b_ws):
        inp = torch.zeros((B,) + in_shape, dtype=dt, device=self.device)
        out = torch.empty((B,) + out_shape, dtype=dt, device=self.device)
        ws = torch.empty(B * b_ws + 256, dtype=torch.uint8, device=self.device)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        # one eager call first: kernel attributes are set outside the capture
        call(plan.handle, B, inp.data_ptr(), out.data_ptr(), ws_ptr, slot.stream.cuda_stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=slot.stream, capture_error_mode="thread_local"):
            call(plan.handle, B, inp.data_ptr(), out.data_ptr(), ws_ptr, slot.stream.cuda_stream)
        nbytes = inp.numel() * inp.element_size() + out.numel() * out.element_size() + ws.numel()
        self.graph_used += nbytes
        return _GraphEntry(g, inp, out, ws, nbytes)

    def _finish(self, slot: _Slot):
        t = time.perf_counter()
        if slot.start is not None:
            self.device_intervals.append((self._ref_event.elapsed_time(slot.start),
                                          self._ref_event.elapsed_time(slot.event), slot.index))
        for i, r in enumerate(slot.batch):
            r.result = slot.out[i]
            r.t_done = t
            self.completed.append(r)
            r.done.set()
        for k in dict.fromkeys(r.key for r in slot.batch):
            self.plan_users[k] -= 1
        self.used -= slot.nbytes
        slot.busy, slot.event, slot.start, slot.batch, slot.buffers, slot.out, slot.nbytes = (False, None, None, [], (),
                                                                                            None, 0)

    # ---------------------------------------------------------------- threads
    def _build_loop(self):
        """Builds the plans that admission asked for, one at a time, without
        holding the server lock."""
        torch.cuda.set_device(self.device)
        while True:
            key = self._build_q.get()
            if key is None:
                return
            mesh, comps, fp64 = key
            try:
                p, err = Plan(mesh, comps, fp64=fp64), None
            except Exception as exc:  # the requests on this plan fail; serving goes on
                p, err = None, f"{type(exc).__name__}: {exc}"
            with self.lock:
                self._build_done(key, p, err)
                self.lock.notify_all()

    def _build_done(self, key, p, err):
        """A build finished (p) or failed (err): swap its reservation for the
        plan's real size, or fail the requests queued on it."""
        self.used -= self.building.pop(key)
        if p is not None:
            self.plans[key] = p
            self.used += p.nbytes
            self.plans_built += 1
        else:
            self._fail_key(key, err)

    def _wait_loop(self, slot: _Slot):
        """Blocks on the completion event of the slot's batch (the thread
        sleeps in the driver, not in a polling loop), then hands the results
        back."""
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                while not slot.busy and not self._stop:
                    self.lock.wait()
                if not slot.busy:
                    return
                ev = slot.event
            ev.synchronize()
            with self.lock:
                self._finish(slot)
                self.lock.notify_all()

    def _loop(self):
        torch.cuda.set_device(self.device)
        with self.lock:
            while True:
                if (self._stop and not self.queue and not self.building
                        and not any(s.busy for s in self.slots)):
                    self.lock.notify_all()
                    return
                progressed = False
                for slot in self.slots:
                    if not self.queue:
                        break
                    if not slot.busy:
                        try:
                            if self._admit(slot):
                                progressed = True
                            else:
                                break
                        except Exception as exc:  # fail the head batch, keep serving
                            head = self.queue.popleft()
                            head.error = f"{type(exc).__name__}: {exc}"
                            head.t_done = time.perf_counter()
                            head.done.set()
                            progressed = True
                if progressed:
                    self.lock.notify_all()  # waiters of the slots just launched
                else:
                    self.lock.wait(0.05)
