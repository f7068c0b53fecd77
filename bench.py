#!/usr/bin/env python
"""Throughput of the fast gravity / gravity-gradient forward on GB300.

One step = one forward of all six components (gz, gxx, gxy, gxz, gyy, gyz)
through the C ABI: row transforms of the density, the fused column stage
(column FFTs, product with the resident FP32 kernel spectra, compensated
layer sum, inverse column FFTs) and inverse row transforms (Eq. 21).

Workload: 1024 x 1024 x 100 cells of 50 x 50 x 25 m, stations 10 m above
the top, density a seeded smooth Gaussian random field (std 200 kg/m^3,
correlation length 20 cells) in float32.  Metric: cell-station pairs per
second, (nx ny) * (nx ny nz) = 1.0995e14 pairs per forward.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs its own replica of
the workload (the forward needs no exchange between ranks); value is the
pairs of all ranks over the slowest rank's time (weak scaling).

``--impl reference`` times the CPU FP64 direct-summation oracle on the
host cores instead, on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (nx, ny, nz, dx, dy, dz, h)
    "grf1024": (1024, 1024, 100, 50.0, 50.0, 25.0, 10.0),
    "grf1024z16": (1024, 1024, 16, 50.0, 50.0, 25.0, 10.0),  # same kernels, fewer layers (profiling)
    "boxes512": (512, 512, 64, 20.0, 20.0, 20.0, 10.0),
    "boxes256": (256, 256, 32, 25.0, 25.0, 20.0, 5.0),
}
METRIC = "6-comp forward cell·station pairs/s at 1024²×100, %HBM roofline; serve p50/p99"
COMPS = 63
NCOMP = 6
FALLBACK_HBM_GBS = 6800.0
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "forward_columns_grf1024.md")
KERNEL_SOURCES = ("fft_block.cuh", "spectral.cuh", "spectral_ws.cuh", "spectral_wf.cuh", "warp_fft.cuh",
                  "spectral_launch.cuh", "async_copy.cuh", "col_fwd_f32.cu", "grav_internal.h")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="grf1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-spectral comparison leg")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests in the serving leg (Poisson arrivals, 0 to skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrival rate of the serving leg (1/s)")
    ap.add_argument("--burst-requests", type=int, default=2000,
                    help="requests in the burst serving leg (2000/s, two station heights; 0 to skip)")
    ap.add_argument("--equal-dim", default="1024,1024,100",
                    help="nx,ny,nz of the equal-dimension leg (grf1024 geometry; 'none' to skip)")
    ap.add_argument("--equal-dim-only", action="store_true",
                    help="run only the equal-dimension leg and print its record (profiling)")
    return ap.parse_args()


def pairs_per_forward(mesh):
    nx, ny, nz = mesh[:3]
    return float(nx * ny) * float(nx * ny * nz)


def kernel_digest() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2005_10160_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(digest: str):
    """DRAM bytes per column-stage launch from the committed ncu summary, or
    None when the summary is missing or the kernel changed since."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_digest") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 100 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((t, float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        window = [r for r in rows if t0 <= r[0] <= t1]
        label = "timed"
        if not window:
            window, label = rows, "warmup+timed"
        if not window:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in window for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in window), "sm_max_mhz": max(r[2] for r in window),
                "reasons": reasons, "samples": len(window), "window": label}


def dist_setup(n_gpus):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """The largest of every rank's value (each rank's timed region; the job
    is as slow as its slowest replica)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step: float, steps: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank (one replica each) runs
    `steps` steps of `units_per_step`, within the slowest rank's time."""
    return world * units_per_step * steps / (ms_max / 1000.0)


def oracle_rate(mesh, rho_np, n_stations, n_layers, threads):
    """Pairs/s of the CPU oracle on n_stations stations x the top n_layers."""
    import numpy as np

    import oracle
    from paper_2005_10160_gb300 import workloads

    nx, ny, nz, dx, dy, dz, h = mesh
    sub = (nx, ny, n_layers, dx, dy, dz, h)
    st = workloads.station_subset(workloads.Mesh(*sub), n_stations, np.random.default_rng(7))
    rho = np.ascontiguousarray(rho_np[:n_layers], dtype=np.float64)
    t0 = time.perf_counter()
    oracle.forward(sub, COMPS, rho, stations=st, nthreads=threads)
    dt = time.perf_counter() - t0
    pairs = float(len(st)) * nx * ny * n_layers
    return pairs / dt, pairs, dt


def cpu_density_sample(mesh, n_layers):
    """The leading layers of the workload's density on the CPU (float32)."""
    import torch

    from paper_2005_10160_gb300 import workloads

    nx, ny, nz = mesh[:3]
    _, rho = workloads.grf1024(nx, ny, nz, device="cuda" if torch.cuda.is_available() else "cpu")
    return rho[:n_layers].float().cpu().numpy()


def serving_leg(n_requests: int, rate: float, heights=(10.0,)):
    """Poisson stream of forward/adjoint requests (50/50) on the four serving
    meshes (64^2x16, 128^2x32, 256^2x32, 512^2x64 of 20 m cubes, random-box
    densities, N(0,1) adjoint inputs), each seen from the given station
    heights, through the continuous-batching server; plans are built during
    a warm-up.  Latency is submission to completion."""
    import numpy as np
    import torch

    from paper_2005_10160_gb300 import workloads
    from paper_2005_10160_gb300.server import Server

    rng = np.random.default_rng(workloads.SEED_BASE + 5)
    meshes = []
    for i in range(4):
        m = workloads.serving_mesh(i)
        meshes += [workloads.Mesh(m.nx, m.ny, m.nz, m.dx, m.dy, m.dz, h) for h in heights]
    pool = {}
    for i, m in enumerate(meshes):
        pool[(i, "forward")] = [torch.as_tensor(workloads.serving_density(m, rng), device="cuda") for _ in range(4)]
        pool[(i, "adjoint")] = [torch.randn((NCOMP, m.ny, m.nx), device="cuda") for _ in range(4)]
    srv = Server(hbm_budget=48 << 30, slots=4, max_batch=8)
    try:
        for i, m in enumerate(meshes):
            for kind in ("forward", "adjoint"):
                srv.submit(kind, m, pool[(i, kind)][0])
        srv.drain()
        srv.completed.clear()
        srv.device_intervals.clear()
        srv.batches_run = srv.graph_replays = srv.cross_plan_batches = srv.max_busy_slots = 0
        t0 = time.perf_counter()
        t_next = t0
        pairs = 0.0
        reqs = []
        swept = 0
        for _ in range(n_requests):
            t_next += float(rng.exponential(1.0 / rate))
            i = int(rng.integers(len(meshes)))
            kind = "forward" if rng.random() < 0.5 else "adjoint"
            m = meshes[i]
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)  # sleeping releases the GIL to the server thread
            reqs.append(srv.submit(kind, m, pool[(i, kind)][int(rng.integers(4))]))
            pairs += pairs_per_forward(m.tuple())
            # results are not needed here: free them as requests finish (only the timings are kept)
            while swept < len(reqs) and reqs[swept].done.is_set():
                reqs[swept].result = None
                swept += 1
        srv.drain()
        for r in reqs:
            r.wait(60)
        st = srv.stats()
        span = max(r.t_done for r in reqs) - t0
    finally:
        srv.close()
    st.update({"rate_per_s": rate, "pairs_per_s": pairs / span,
               "workload": "Poisson 50/50 forward/adjoint on 64^2x16, 128^2x32, 256^2x32, 512^2x64 (20 m cubes), "
                           f"stations {', '.join(f'{h:g}' for h in heights)} m up, FP32 spectra, plans resident"})
    return st


def equal_dim_leg(dims: str, dev, peak: float):
    """Forward and adjoint of the equal-dimension variant (a station at the
    centre of every cell) on the grf1024 geometry (50 x 50 x 25 m cells) with
    the smooth random-field density, six components, FP32 spectra; device
    time by CUDA events.  Method bytes: the stored three-level spectra + rho +
    the six output volumes."""
    import torch

    from paper_2005_10160_gb300 import workloads
    from paper_2005_10160_gb300.plan import Plan3D

    nx, ny, nz = (int(v) for v in dims.split(","))
    mesh, rho = workloads.grf1024(nx, ny, nz, device=dev)
    rho = rho.contiguous()
    t0 = time.perf_counter()
    plan = Plan3D(mesh, COMPS, fp64=False)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    out = torch.empty((NCOMP, nz, ny, nx), dtype=torch.float32, device=dev)
    grad = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        plan.forward(rho, out)
        plan.adjoint(out, grad)
    torch.cuda.synchronize()
    n = 5
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(n):
        plan.forward(rho, out)
    e1.record(stream)
    for _ in range(n):
        plan.adjoint(out, grad)
    e2.record(stream)
    torch.cuda.synchronize()
    f_ms = e0.elapsed_time(e1) / n
    a_ms = e1.elapsed_time(e2) / n
    cells = float(nx * ny * nz)
    pairs = cells * cells
    method = plan.spectra_bytes + 4 * cells + 4 * NCOMP * cells
    res = {"workload": f"equal-dimension {nx}x{ny}x{nz} cells 50x50x25 m, a station at every cell centre, "
                       f"{NCOMP} components, FP32 spectra, smooth random-field density",
           "pairs_per_forward": pairs, "plan_create_s": plan_s, "pz": plan.pz,
           "forward_ms": f_ms, "forward_pairs_per_s": pairs / (f_ms / 1000.0),
           "adjoint_ms": a_ms, "adjoint_pairs_per_s": pairs / (a_ms / 1000.0),
           "method_bytes": method, "spectra_bytes": plan.spectra_bytes,
           "forward_frac": method / (f_ms / 1000.0) / 1e9 / peak,
           "adjoint_frac": method / (a_ms / 1000.0) / 1e9 / peak,
           "frac_what": "(stored spectra + rho + out) / device time / measured HBM copy bandwidth"}
    plan.close()
    return res


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    mesh = WORKLOADS[args.workload]
    cores = os.cpu_count() or 1
    rho = cpu_density_sample(mesh, mesh[2])
    # calibrate, then size each step to keep the whole run within ~2.5 minutes
    rate0, _, _ = oracle_rate(mesh, rho, cores, 1, cores)
    per_step_s = 150.0 / max(1, args.steps + args.warmup)
    layers = int(max(1, min(mesh[2], per_step_s * rate0 / (cores * mesh[0] * mesh[1]))))
    for _ in range(args.warmup):
        oracle_rate(mesh, rho, cores, layers, cores)
    tot_pairs = tot_s = 0.0
    for _ in range(args.steps):
        _, p, dt = oracle_rate(mesh, rho, cores, layers, cores)
        tot_pairs += p
        tot_s += dt
    value = tot_pairs / tot_s
    sample = f"{cores} stations x top {layers} of {mesh[2]} layers x {mesh[0]}x{mesh[1]} cells per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} {mesh[0]}x{mesh[1]}x{mesh[2]}, {NCOMP} components",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    if args.equal_dim_only:
        from paper_2005_10160_gb300 import build as gbuild
        from paper_2005_10160_gb300 import capi

        gbuild.build()
        capi.lib()
        torch.cuda.set_device(0)
        print(json.dumps({"equal_dim": equal_dim_leg(args.equal_dim, torch.device("cuda", 0), hbm_peak()[0])}),
              flush=True)
        return 0

    from paper_2005_10160_gb300 import build as gbuild
    from paper_2005_10160_gb300 import capi, workloads
    from paper_2005_10160_gb300.pipeline import HostPipeline
    from paper_2005_10160_gb300.plan import Plan

    world, rank, local = dist_setup(args.gpus)
    if rank == 0:
        gbuild.build()
    barrier(world)
    capi.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    mesh = WORKLOADS[args.workload]
    nx, ny, nz = mesh[:3]
    pairs = pairs_per_forward(mesh)

    if args.workload.startswith("grf1024"):
        _, rho = workloads.grf1024(nx, ny, nz, device=dev)
    else:
        m = workloads.Mesh(*mesh)
        rho = torch.as_tensor(workloads.serving_density(m, workloads.rng_for(9)), device=dev)
    rho = rho.to(torch.float32).contiguous()

    t0 = time.perf_counter()
    plan = Plan(mesh, COMPS, fp64=False)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    out = torch.empty((NCOMP, ny, nx), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) > 8:
        gpu_id = "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id)
    sampler.start()

    for _ in range(args.warmup):
        plan.forward(rho, out)
    torch.cuda.synchronize()
    capi.grav_plan_set_timing(plan.handle, True)
    capi.grav_plan_stage_times(plan.handle)  # reset

    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        plan.forward(rho, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    stage_ms, n_fwd, _ = capi.grav_plan_stage_times(plan.handle)
    capi.grav_plan_set_timing(plan.handle, False)
    ms_max = max_over_ranks(world, ms)
    sampler.stop()
    clocks = sampler.summary(t_wall0 - 0.05, t_wall1 + 0.05)

    ms_per_step = ms_max / args.steps
    value = whole_job_rate(world, pairs, args.steps, ms_max)

    # roofline of the dominant kernel, the column stage, on the method's own
    # bytes: the stored kernel spectra it streams once (one FP32 real per
    # (kx, mirror pair, layer, component); they replace G, Eq. 22)
    kx = plan.px // 2 + 1
    hy = plan.py // 2 + 1
    spec_b = NCOMP * nz * kx * hy * 4
    x_b = kx * nz * ny * 8          # row transforms of rho, read (implementation traffic)
    y_b = 2 * kx * NCOMP * ny * 8   # column outputs, written (implementation traffic)
    col_ms = stage_ms["forward_columns"] / max(1, n_fwd)
    peak, peak_kind = hbm_peak()
    achieved = spec_b / (col_ms / 1000.0) / 1e9
    digest = kernel_digest()
    traffic = profiled_traffic(digest)
    fwd_alg = spec_b + 4 * nx * ny * nz + 4 * NCOMP * nx * ny  # spectra + rho + out
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "forward_column_wf_kernel<6> (column stage)",
                "algorithmic_bytes": spec_b, "avg_launch_ms": col_ms, "peak_kind": peak_kind,
                "dram_efficiency": {"bytes": spec_b + x_b + y_b,
                                    "frac": (spec_b + x_b + y_b) / (col_ms / 1000.0) / 1e9 / peak,
                                    "what": "spectra + row transforms read + column outputs written, per launch"},
                "whole_forward": {"bytes": fwd_alg, "ms": ms_per_step,
                                  "frac": fwd_alg / (ms_per_step / 1000.0) / 1e9 / peak,
                                  "what": "stored spectra + rho + out over the device time of one forward"},
                "stage_ms": {k: v / max(1, n_fwd) for k, v in stage_ms.items() if k.startswith("forward")}}

    # end to end through the public API with pinned host buffers
    rho_h = rho.cpu().pin_memory()
    out_h = torch.empty((NCOMP, ny, nx), dtype=torch.float32).pin_memory()
    rho_d = torch.empty_like(rho)
    for _ in range(max(1, args.warmup)):
        rho_d.copy_(rho_h, non_blocking=True)
        plan.forward(rho_d, out)
        out_h.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e_steps = max(3, min(args.steps, 50))
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e_steps):
        rho_d.copy_(rho_h, non_blocking=True)
        plan.forward(rho_d, out)
        out_h.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e_ms = max_over_ranks(world, e0.elapsed_time(e1))
    seq_ms = e_ms / e_steps

    # the same with HostPipeline (two lanes): step i+1's host-to-device copy
    # overlaps step i's kernels; every step still copies its own density in
    # and its own six planes out
    pipe = HostPipeline(plan, lanes=2)
    outs_h = [torch.empty((NCOMP, ny, nx), dtype=torch.float32).pin_memory() for _ in pipe.lanes]
    for i in range(max(2, args.warmup)):
        pipe.forward(rho_h, outs_h[i % 2])
    pipe.synchronize()
    barrier(world)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(e_steps):
        pipe.forward(rho_h, outs_h[i % 2], after=start if i < 2 else None)
    pipe.join(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    p_ms = max_over_ranks(world, start.elapsed_time(stop))
    e2e = {"value": whole_job_rate(world, pairs, e_steps, p_ms), "unit": "pairs/s",
           "h2d_bytes_per_step": rho_h.numel() * 4, "d2h_bytes_per_step": out_h.numel() * 4,
           "steps": e_steps, "ms_per_step": p_ms / e_steps,
           "mode": "HostPipeline, 2 lanes (copies of one step overlap the kernels of the previous)",
           "sequential_ms_per_step": seq_ms}
    del pipe

    # the adjoint G^T r on the same plan (HBM-bound like the forward: it streams
    # every spectrum once), device-resident N(0,1) residual planes
    gen = torch.Generator(device=dev)
    gen.manual_seed(20051016 + 3)
    r_in = torch.randn((NCOMP, ny, nx), dtype=torch.float32, device=dev, generator=gen)
    grad = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.adjoint(r_in, grad)
    torch.cuda.synchronize()
    capi.grav_plan_set_timing(plan.handle, True)
    capi.grav_plan_stage_times(plan.handle)  # reset
    a_steps = max(3, min(args.steps, 20))
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(a_steps):
        plan.adjoint(r_in, grad)
    a1.record(stream)
    torch.cuda.synchronize()
    a_stage, _, n_adj = capi.grav_plan_stage_times(plan.handle)
    capi.grav_plan_set_timing(plan.handle, False)
    a_ms = max_over_ranks(world, a0.elapsed_time(a1)) / a_steps
    a_col_ms = a_stage["adjoint_columns"] / max(1, n_adj)
    adj_alg = spec_b + 4 * NCOMP * nx * ny + 4 * nx * ny * nz  # spectra + r + grad
    adjoint = {"ms_per_step": a_ms, "value": whole_job_rate(world, pairs, 1, a_ms), "unit": "pairs/s", "steps": a_steps,
               "stage_ms": {k: v / max(1, n_adj) for k, v in a_stage.items() if k.startswith("adjoint")},
               "column_stage_frac": spec_b / (a_col_ms / 1000.0) / 1e9 / peak,
               "whole_adjoint_frac": adj_alg / (a_ms / 1000.0) / 1e9 / peak}
    del r_in, grad

    # the all-FP64 spectral path on the same workload, for context
    fp64 = None
    if not args.no_fp64 and rank == 0:
        plan64 = Plan(mesh, COMPS, fp64=True)
        rho64 = rho.double()
        out64 = torch.empty((NCOMP, ny, nx), dtype=torch.float64, device=dev)
        plan64.forward(rho64, out64)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        n64 = 3
        for _ in range(n64):
            plan64.forward(rho64, out64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / n64
        diff = (out.double() - out64).reshape(NCOMP, -1)
        rel = (torch.linalg.vector_norm(diff, dim=1)
               / torch.linalg.vector_norm(out64.reshape(NCOMP, -1), dim=1)).cpu().tolist()
        units = torch.tensor([1e5] + [1e9] * (NCOMP - 1), dtype=torch.float64, device=dev)  # mGal, Eotvos
        maxabs = (diff.abs().amax(dim=1) * units).cpu().tolist()
        peak_val = (out64.reshape(NCOMP, -1).abs().amax(dim=1) * units).cpu().tolist()
        fp64 = {"ms_per_step": ms64, "value": pairs / (ms64 / 1000.0),
                "fp32_vs_fp64_rel_l2": rel, "fp32_vs_fp64_max_abs_mgal_eotvos": maxabs,
                "field_max_abs_mgal_eotvos": peak_val,
                "components": ["gz (mGal)", "gxx (E)", "gxy (E)", "gxz (E)", "gyy (E)", "gyz (E)"]}
        plan64.close()
        del rho64, out64

    # the full inversion loop (damped CGLS with depth weights) on the 512^2 x 64
    # three-box model, gz + gzz data with 1% noise: one forward and one adjoint
    # per iteration through the C ABI
    inversion = None
    if rank == 0 and args.workload == "grf1024":
        from paper_2005_10160_gb300.inversion import cg_step, cgls, noisy_data

        imesh, irho, _ = workloads.boxes512()
        icomps = capi.GRAV_GZ | capi.GRAV_GZZ
        with Plan(imesh, icomps) as ip:
            clean = ip.forward(torch.as_tensor(irho, dtype=torch.float32, device=dev))
            d_i, w_i = noisy_data(clean.cpu(), 0.01, seed=workloads.SEED_BASE + 4)
            d_i, w_i = d_i.to(dev), w_i.to(dev)
            lam_i = cg_step(ip, d_i, w_i).lam
            cgls(ip, d_i, w_i, lam_i, iters=2)  # warm-up
            res = cgls(ip, d_i, w_i, lam_i, iters=10)
        inversion = {"workload": "512x512x64 cubes of 20 m, three boxes, gz + gzz data with 1% noise, "
                                 "depth weights beta = 2, damped CGLS",
                     "iterations": res.iterations, "ms_per_iteration": res.ms_per_iteration,
                     "lam": res.lam, "objective_first": res.objectives[0], "objective_last": res.objectives[-1]}

    # the equal-dimension variant (a station at every cell centre, Eqs. 10-11)
    equal_dim = None
    if rank == 0 and args.equal_dim != "none":
        plan.close()
        equal_dim = equal_dim_leg(args.equal_dim, dev, peak)

    serving = None
    if rank == 0 and args.serve_requests > 0:
        plan.close()
        serving = serving_leg(args.serve_requests, args.serve_rate)
        if args.burst_requests > 0:
            serving = {**serving, "burst": serving_leg(args.burst_requests, 2000.0, heights=(10.0, 50.0))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "grf1024":
        cores = os.cpu_count() or 1
        layers = 16
        rho_np = rho[:layers].cpu().numpy()
        rate, p, dt = oracle_rate(mesh, rho_np, cores, layers, cores)
        cpu = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": f"{cores} stations x top {layers} layers x {nx}x{ny} cells ({p:.3g} pairs, {dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload} {nx}x{ny}x{nz} cells {mesh[3]:g}x{mesh[4]:g}x{mesh[5]:g} m, "
                                   f"h={mesh[6]:g} m, {NCOMP} components, FP32 spectra",
                       "pairs_per_step": pairs, "l2": "inputs larger than L2 (spectra %.2f GB)" % (spec_b / 1e9),
                       "parallelism": f"replica x{world}", "plan_create_s": plan_s,
                       "forward_algorithmic_bytes": fwd_alg},
            "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": 3 * args.steps,
            "cpu_baseline": cpu, "fp64_path": fp64, "adjoint": adjoint, "inversion": inversion, "serving": serving,
            "equal_dim": equal_dim,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
