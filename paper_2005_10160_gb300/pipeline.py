"""Forwards on host-resident inputs with the copies of one request overlapping
the kernels of the previous one.

A plan's own workspaces serve one call at a time.  HostPipeline keeps
`lanes` independent lanes, each with its own CUDA stream, batched-call
workspace (BatchRunner, grav_forward_batch with a count of 1) and device
buffers for the density and the result.  Request i runs on lane i % lanes:
the host-to-device copy of its density, the forward, and the device-to-host
copy of its result are queued on that lane's stream, so while one lane's
kernels run, the next lane's copy engine traffic proceeds.  Every request
still moves its own input in and its own result out.

Host buffers must be pinned (torch.Tensor.pin_memory()) for the copies to be
asynchronous; a result buffer may be read once the event returned by
forward() has completed.
"""
from __future__ import annotations

import torch

from .batch import BatchRunner
from .plan import Plan


class _Lane:
    def __init__(self, plan: Plan):
        nx, ny, nz = plan.mesh[:3]
        self.stream = torch.cuda.Stream(device=plan.device)
        self.runner = BatchRunner(plan)
        self.rho = torch.empty((1, nz, ny, nx), dtype=plan.dtype, device=plan.device)
        self.out = torch.empty((1, plan.ncomp, ny, nx), dtype=plan.dtype, device=plan.device)
        self.done = torch.cuda.Event()


class HostPipeline:
    def __init__(self, plan: Plan, lanes: int = 2):
        if lanes < 1:
            raise ValueError("lanes must be >= 1")
        self.plan = plan
        self.lanes = [_Lane(plan) for _ in range(lanes)]
        self.count = 0

    def forward(self, rho_host: torch.Tensor, out_host: torch.Tensor, after: torch.cuda.Event | None = None):
        """Queue one forward: rho_host [nz][ny][nx] (pinned) -> out_host
        [ncomp][ny][nx] (pinned).  `after`: an event the lane waits for first.
        Returns the event that marks the result as copied out."""
        lane = self.lanes[self.count % len(self.lanes)]
        self.count += 1
        if after is not None:
            lane.stream.wait_event(after)
        with torch.cuda.stream(lane.stream):
            lane.rho[0].copy_(rho_host, non_blocking=True)
            lane.runner.forward(lane.rho, lane.out, stream=lane.stream)
            out_host.copy_(lane.out[0], non_blocking=True)
            lane.done.record(lane.stream)
        return lane.done

    def join(self, stream: torch.cuda.Stream | None = None) -> None:
        """Make `stream` (default: the current stream) wait for every queued request."""
        s = stream if stream is not None else torch.cuda.current_stream(self.plan.device)
        for lane in self.lanes:
            s.wait_event(lane.done)

    def synchronize(self) -> None:
        for lane in self.lanes:
            lane.stream.synchronize()
