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

``cgls`` runs the full inversion loop: the same Tikhonov problem with depth
weights on the model,
    min_m  ||W (G m - d)||^2 + lam ||W_m m||^2,
W_m = diag(w_n), w_n = (h + (n + 1/2) dz)^(-beta/2) per layer (Li and
Oldenburg 1996: undoes the decay of the kernel with depth, so that the
recovered density is not pushed to the surface), scaled to max 1, solved by
conjugate gradients on the normal equations in x = W_m m (damped CGLS:
Hestenes and Stiefel 1952, Bjorck 1996).  Every iteration is one forward
and one adjoint through the C ABI; the vector updates are elementwise
device operations with FP64 reductions.
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


def depth_weights(mesh, beta: float = 2.0, device=None, dtype=torch.float32) -> torch.Tensor:
    """w_n = (h + (n + 1/2) dz)^(-beta/2), scaled to max 1, shaped [nz, 1, 1]."""
    nz, dz, h = int(mesh[2]), float(mesh[5]), float(mesh[6])
    z = h + (torch.arange(nz, dtype=torch.float64) + 0.5) * dz
    w = z.pow(-beta / 2.0)
    return (w / w.max()).to(device=device, dtype=dtype)[:, None, None]


@dataclass
class CGLSResult:
    m: torch.Tensor           # model after the last iteration [nz][ny][nx]
    models: list              # model after each iteration (if kept)
    objectives: list          # J(m_k), k = 0 .. iterations (from the recurrence residual)
    iterations: int
    lam: float
    ms_per_iteration: float   # CUDA-event time of one iteration (forward + adjoint + updates)


def _dot(a: torch.Tensor, b: torch.Tensor) -> float:
    return float(torch.sum(a * b, dtype=torch.float64))


def cgls(plan: Plan, d: torch.Tensor, w: torch.Tensor, lam: float, iters: int = 10, beta: float = 2.0,
         keep_models: bool = False) -> CGLSResult:
    """Damped CGLS with depth weights (see the module docstring).

    d: data [ncomp][ny][nx]; w: data weights broadcastable to d (1/sigma_c as
    [ncomp, 1, 1]); lam: Tikhonov weight on ||W_m m||^2; iters: iterations.
    plan: anything with .mesh, .forward and .adjoint on d's device (a Plan).
    Returns the model m = W_m^-1 x and the objective after every iteration;
    ms_per_iteration is timed with CUDA events when d is on a GPU (else nan)."""
    wm = depth_weights(plan.mesh, beta, device=d.device, dtype=d.dtype)

    def A(x):
        return w * plan.forward((x / wm).contiguous())

    def At(r):
        return plan.adjoint((w * r).contiguous()) / wm

    b = (w * d).contiguous()
    x = torch.zeros((plan.mesh[2], plan.mesh[1], plan.mesh[0]), dtype=d.dtype, device=d.device)
    r = b.clone()
    s = At(r)
    p = s.clone()
    gamma = _dot(s, s)
    objectives = [_dot(r, r)]
    models = []
    timed = d.is_cuda
    if timed:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
    for _ in range(iters):
        if gamma == 0.0:
            objectives.append(objectives[-1])
            if keep_models:
                models.append((x / wm).clone())
            continue
        q = A(p)
        alpha = gamma / (_dot(q, q) + lam * _dot(p, p))
        x.add_(p, alpha=alpha)
        r.sub_(q, alpha=alpha)
        s = At(r)
        s.sub_(x, alpha=lam)
        gamma_new = _dot(s, s)
        p.mul_(gamma_new / gamma).add_(s)
        gamma = gamma_new
        objectives.append(_dot(r, r) + lam * _dot(x, x))
        if keep_models:
            models.append((x / wm).clone())
    ms = float("nan")
    if timed:
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(1, iters)
    return CGLSResult(m=x / wm, models=models, objectives=objectives, iterations=iters, lam=lam,
                      ms_per_iteration=ms)


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
