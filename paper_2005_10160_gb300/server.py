"""Continuous-batching request loop over resident plans.

Forward and adjoint requests on meshes of different sizes arrive at any
time.  The loop keeps each mesh's plan (its kernel spectra, Eq. 22) resident
on the device, admits queued requests into execution slots as slots and
device memory free up, groups queued requests on the same plan and of the
same kind into one batched call (one launch per stage for the whole
batch), runs each slot on its own CUDA stream so that work of different
slots overlaps on the GPU, and records per-request latency from submission
to the completion of its batch on the device.

Admission is by an HBM budget: resident plans plus, for every batch in
flight, its input, output and workspace buffers.  A plan that is not in use
may be evicted (least recently used) to admit another.  Small batches are
replayed from CUDA graphs captured per (slot, plan, kind, batch size).

All arithmetic happens in libgravfft.so through the C ABI.
"""
from __future__ import annotations

import collections
import itertools
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
    requests per batched call.  graph_bytes_limit: per-request size (input +
    output + workspace) below which batches are replayed from CUDA graphs."""

    def __init__(self, hbm_budget: int, slots: int = 4, max_batch: int = 8, device=None,
                 graph_bytes_limit: int = 64 << 20, graph_memory: int = 2 << 30):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.graph_bytes_limit = int(graph_bytes_limit)
        self.graph_memory = int(graph_memory)
        self.plans: "collections.OrderedDict[tuple, Plan]" = collections.OrderedDict()
        self.plan_users: dict[tuple, int] = collections.defaultdict(int)
        self.used = 0
        self.graph_used = 0
        self.queue: collections.deque[Request] = collections.deque()
        self.lock = threading.Condition()
        self.slots = [_Slot(self.device, i) for i in range(slots)]
        self.ids = itertools.count()
        self.completed: list[Request] = []
        self.batches_run = 0
        self.graph_replays = 0
        self.max_busy_slots = 0
        # device time line: every batch's [start, end] in ms after the
        # reference event, from events on the slot streams (one GPU clock)
        self.device_intervals: list[tuple[float, float, int]] = []
        self._ref_event = torch.cuda.Event(enable_timing=True)
        with torch.cuda.device(self.device):
            self._ref_event.record(torch.cuda.current_stream(self.device))
        self._stop = False
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
            self.lock.notify()
        return req

    def drain(self, timeout: float = 300.0):
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.lock:
            while self.queue or any(s.busy for s in self.slots):
                if time.perf_counter() - t0 > timeout:
                    raise TimeoutError("server did not drain")
                self.lock.wait(0.01)

    def close(self):
        self.drain()
        with self.lock:
            self._stop = True
            self.lock.notify()
        self._thread.join()
        for slot in self.slots:
            slot.graphs.clear()
        for p in self.plans.values():
            p.close()
        self.plans.clear()

    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.completed if r.error is None])
        if lat.size == 0:
            return {"requests": 0}
        span = max(r.t_done for r in self.completed) - min(r.t_submit for r in self.completed)
        return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                "req_per_s": float(lat.size / span) if span > 0 else None, "batches": self.batches_run,
                "graph_replays": self.graph_replays, "max_busy_slots": self.max_busy_slots,
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
    def _plan(self, key) -> Plan | None:
        """Resident plan for key, created (evicting idle plans) if needed;
        None while the budget cannot hold it yet."""
        if key in self.plans:
            self.plans.move_to_end(key)
            return self.plans[key]
        mesh, comps, fp64 = key
        need = self._plan_bytes_estimate(mesh, comps, fp64)
        while self.used + need > self.budget:
            idle = [k for k in self.plans if self.plan_users[k] == 0]
            if not idle:
                return None
            victim = idle[0]
            p = self.plans.pop(victim)
            self.used -= p.nbytes
            for slot in self.slots:
                for gk in [g for g in slot.graphs if g[0] == victim]:
                    self.graph_used -= slot.graphs.pop(gk).nbytes
            p.close()
        with torch.cuda.device(self.device):
            p = Plan(mesh, comps, fp64=fp64)
        self.plans[key] = p
        self.used += p.nbytes
        return p

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

    def _take_batch(self):
        """Oldest request plus later queued ones on the same plan and kind."""
        head = self.queue[0]
        batch = [head]
        for r in itertools.islice(self.queue, 1, None):
            if len(batch) >= self.max_batch:
                break
            if r.key == head.key and r.kind == head.kind:
                batch.append(r)
        return batch

    def _admit(self, slot: _Slot) -> bool:
        batch = self._take_batch()
        key, kind = batch[0].key, batch[0].kind
        plan = self._plan(key)
        if plan is None:
            if any(s.busy for s in self.slots):
                return False  # a batch in flight may release its plan
            need = self._plan_bytes_estimate(*key)
            for r in batch:
                self.queue.remove(r)
                r.error = f"the plan needs {need} bytes beyond the HBM budget of {self.budget}"
                r.t_done = time.perf_counter()
                r.done.set()
            return True
        b_in, b_out, b_ws = self._request_bytes(plan, kind)
        per_req = b_in + b_out + b_ws
        use_graph = per_req <= self.graph_bytes_limit
        gkey = (key, kind, len(batch))
        # a graph replay needs only the cloned output; an eager batch its buffers
        need = len(batch) * (b_out if (use_graph and gkey in slot.graphs) else per_req)
        if self.used + self.graph_used + need > self.budget:
            if any(s.busy for s in self.slots):
                return False  # wait for a batch in flight to release memory
            # nothing in flight will free memory: drop captured graphs and idle
            # plans, then fail the batch if it still does not fit
            for s in self.slots:
                for g in list(s.graphs):
                    self.graph_used -= s.graphs.pop(g).nbytes
            for k in [k for k in self.plans if k != key and self.plan_users[k] == 0]:
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
        self.plan_users[key] += 1
        self._launch(slot, plan, kind, batch, use_graph, (b_in, b_out, b_ws))
        return True

    def _launch(self, slot: _Slot, plan: Plan, kind: str, batch: list[Request], use_graph: bool, sizes):
        b_in, b_out, b_ws = sizes
        B = len(batch)
        nx, ny, nz = plan.mesh[:3]
        out_shape = (nz, ny, nx) if kind == "adjoint" else (plan.ncomp, ny, nx)
        in_shape = tuple(batch[0].data.shape)
        dt = plan.dtype
        call = capi.grav_forward_batch if kind == "forward" else capi.grav_adjoint_batch
        gkey = (batch[0].key, kind, B)
        with torch.cuda.device(self.device), torch.cuda.stream(slot.stream):
            for r in batch:  # inputs were produced on the submitting thread's stream
                slot.stream.wait_event(r.ready)
                r.data.record_stream(slot.stream)
            start = torch.cuda.Event(enable_timing=True)
            start.record(slot.stream)
            if use_graph:
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
            if not use_graph:
                inp = torch.stack([r.data for r in batch])
                out = torch.empty((B,) + out_shape, dtype=dt, device=self.device)
                ws = torch.empty(B * b_ws + 256, dtype=torch.uint8, device=self.device)
                ws_ptr = (ws.data_ptr() + 255) // 256 * 256
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
        self.plan_users[slot.batch[0].key] -= 1
        self.used -= slot.nbytes
        slot.busy, slot.event, slot.start, slot.batch, slot.buffers, slot.out, slot.nbytes = (False, None, None, [], (),
                                                                                            None, 0)

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            progressed = False
            with self.lock:
                for slot in self.slots:
                    if slot.busy and slot.event.query():
                        self._finish(slot)
                        progressed = True
                if self._stop and not self.queue and not any(s.busy for s in self.slots):
                    self.lock.notify_all()
                    return
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
                self.lock.notify_all()
                if not progressed:
                    self.lock.wait(0.0002)
