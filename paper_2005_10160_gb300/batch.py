"""Batched forward and adjoint on one plan with a caller-owned workspace
(grav_forward_batch / grav_adjoint_batch): one launch per stage for a whole
batch of independent requests on the same mesh."""
from __future__ import annotations

import torch

from . import capi
from .plan import Plan


class BatchRunner:
    """Holds a workspace sized for up to ``capacity`` requests (grown on
    demand) so that batched calls on its stream do not share the plan's own
    workspaces."""

    def __init__(self, plan: Plan, capacity: int = 1):
        self.plan = plan
        self.per_request = capi.grav_workspace_bytes(plan.handle)
        self._ws = None
        self._reserve(capacity)

    def _reserve(self, batch: int):
        need = batch * self.per_request + 256
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.plan.device)

    def _ws_ptr(self) -> int:
        return (self._ws.data_ptr() + 255) // 256 * 256

    def forward(self, rho: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """rho [batch][nz][ny][nx] -> [batch][ncomp][ny][nx]."""
        nx, ny, nz = self.plan.mesh[:3]
        b = rho.shape[0]
        if tuple(rho.shape[1:]) != (nz, ny, nx) or rho.dtype != self.plan.dtype or not rho.is_contiguous():
            raise ValueError("rho must be contiguous [batch][nz][ny][nx] of the plan's dtype")
        if out is None:
            out = torch.empty((b, self.plan.ncomp, ny, nx), dtype=self.plan.dtype, device=self.plan.device)
        self._reserve(b)
        s = stream if stream is not None else torch.cuda.current_stream(self.plan.device)
        capi.grav_forward_batch(self.plan.handle, b, rho.data_ptr(), out.data_ptr(), self._ws_ptr(), s.cuda_stream)
        return out

    def adjoint(self, r: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """r [batch][ncomp][ny][nx] -> [batch][nz][ny][nx]."""
        nx, ny, nz = self.plan.mesh[:3]
        b = r.shape[0]
        if tuple(r.shape[1:]) != (self.plan.ncomp, ny, nx) or r.dtype != self.plan.dtype or not r.is_contiguous():
            raise ValueError("r must be contiguous [batch][ncomp][ny][nx] of the plan's dtype")
        if out is None:
            out = torch.empty((b, nz, ny, nx), dtype=self.plan.dtype, device=self.plan.device)
        self._reserve(b)
        s = stream if stream is not None else torch.cuda.current_stream(self.plan.device)
        capi.grav_adjoint_batch(self.plan.handle, b, r.data_ptr(), out.data_ptr(), self._ws_ptr(), s.cuda_stream)
        return out
