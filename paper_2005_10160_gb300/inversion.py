"""Differentiation through the fast forward and one step of least-squares
density inversion (the forward model is the inner loop of inversion,
Sec. 1 and Sec. 4).

``GravForward`` is a torch.autograd.Function whose backward is the adjoint
G^T (the transpose of Eq. 21: a per-layer product with the conjugate kernel
spectra and no sum over layers), so gradients never need G itself.

``cg_step`` takes one conjugate-gradient step of the Tikhonov problem
    min_m  J(m) = ||W (G m - d)||^2 + lam ||m||^2
from m0 = 0: the first CG direction is the negative gradient
g = G^T W^2 d, and the exact line search along it gives
    m1 = ||g||^2 / (||W G g||^2 + lam ||g||^2) * g.
Both products run through the C ABI (forward and adjoint).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from .plan import Plan


class GravForward(torch.autograd.Function):
    """d = G rho through the plan; backward applies G^T."""

    @staticmethod
    def forward(ctx, rho: torch.Tensor, plan: Plan) -> torch.Tensor:
        ctx.plan = plan
        return plan.forward(rho.contiguous())

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        return ctx.plan.adjoint(grad_out.contiguous()), None


def forward_model(rho: torch.Tensor, plan: Plan) -> torch.Tensor:
    return GravForward.apply(rho, plan)


@dataclass
class CGStep:
    m1: torch.Tensor      # updated model [nz][ny][nx]
    g: torch.Tensor       # first direction G^T W^2 d
    alpha: float          # step length
    lam: float            # Tikhonov weight used
    J0: float             # objective at m = 0
    J1: float             # objective at m1


def objective(plan: Plan, m: torch.Tensor, d: torch.Tensor, w: torch.Tensor, lam: float) -> float:
    r = w * (plan.forward(m) - d)
    return float((r.double() ** 2).sum() + lam * (m.double() ** 2).sum())


def cg_step(plan: Plan, d: torch.Tensor, w: torch.Tensor, lam: float | None = None,
            lam_rel: float = 1e-2) -> CGStep:
    """One CG step from m0 = 0.

    d: data [ncomp][ny][nx]; w: per-component weights broadcastable to d
    (e.g. 1/sigma_c with shape [ncomp, 1, 1]); lam: Tikhonov weight, or
    lam_rel * ||W G g||^2 / ||g||^2 when None."""
    w2d = (w * w * d).contiguous()
    g = plan.adjoint(w2d)
    Gg = plan.forward(g)
    gg = float((g.double() ** 2).sum())
    wGg = float(((w * Gg).double() ** 2).sum())
    if lam is None:
        lam = lam_rel * wGg / gg
    alpha = gg / (wGg + lam * gg)
    m1 = (alpha * g.double()).to(g.dtype)
    J0 = float(((w * d).double() ** 2).sum())
    J1 = objective(plan, m1, d, w, lam)
    return CGStep(m1=m1, g=g, alpha=alpha, lam=lam, J0=J0, J1=J1)


def noisy_data(clean: torch.Tensor, rel_noise: float, seed: int):
    """Data with Gaussian noise of rel_noise times each component's RMS, and
    the weights 1/sigma_c.  clean: [ncomp][ny][nx]."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    rms = clean.double().pow(2).mean(dim=(1, 2)).sqrt()
    sigma = rel_noise * rms
    noise = torch.randn(clean.shape, generator=gen, dtype=torch.float64) * sigma.cpu()[:, None, None]
    d = (clean.double() + noise.to(clean.device)).to(clean.dtype)
    w = (1.0 / sigma).to(clean.dtype)[:, None, None]
    return d, w
