"""Differentiation form: the adjoint behind torch.autograd, finite
differences on 64 random cells of the 512 x 512 x 64 mesh, and one CG step
of Tikhonov least squares on gz + gzz data (1% noise), against the oracle's
explicit G at a tiny size and against the FP64 path at full size."""
import numpy as np
import pytest
import torch

from paper_2005_10160_gb300 import capi, workloads as W
from paper_2005_10160_gb300.inversion import cg_step, cgls, forward_model, noisy_data
from paper_2005_10160_gb300.plan import Plan

pytestmark = pytest.mark.gpu

DATA_COMPS = capi.GRAV_GZ | capi.GRAV_GZZ


def test_autograd_backward_is_the_adjoint(gravlib, orc):
    mesh = (9, 7, 4, 10.0, 12.0, 8.0, 2.0)
    rng = np.random.default_rng(1)
    rho = torch.tensor(rng.uniform(-300, 300, (4, 7, 9)), dtype=torch.float64, device="cuda", requires_grad=True)
    r = rng.normal(size=(6, 7, 9))
    with Plan(mesh, capi.GRAV_ALL6, fp64=True) as plan:
        d = forward_model(rho, plan)
        (d * torch.as_tensor(r, device="cuda")).sum().backward()
    ref = orc.adjoint(mesh, capi.GRAV_ALL6, r)
    got = rho.grad.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_finite_differences_on_64_cells(gravlib):
    """(F(m + e_j) - F(m - e_j)) / 2 dotted with r equals (G^T r)_j.  The map is
    linear, so the difference quotient is the same at every base point m and
    exact up to round-off; m = 0 keeps the two fields from cancelling (the
    difference of two full fields of the model would lose the single cell's
    contribution in round-off)."""
    mesh, rho, _ = W.boxes512()
    nz, ny, nx = rho.shape
    rng = np.random.default_rng(64)
    cells = rng.choice(nz * ny * nx, size=64, replace=False)
    for fp64 in (True, False):
        dt = torch.float64 if fp64 else torch.float32
        with Plan(mesh, capi.GRAV_ALL6, fp64=fp64) as plan:
            r = torch.as_tensor(rng.normal(size=(6, ny, nx)), dtype=dt, device="cuda")
            adj = plan.adjoint(r).reshape(-1)
            base = torch.zeros((nz, ny, nx), dtype=dt, device="cuda")
            eps = 1.0
            for j in cells:
                e = torch.zeros(nz * ny * nx, dtype=dt, device="cuda")
                e[j] = eps
                fp = plan.forward(base + e.reshape(nz, ny, nx))
                fm = plan.forward(base - e.reshape(nz, ny, nx))
                diff = ((fp - fm) / (2 * eps)).double()
                fd = float((diff * r.double()).sum())
                scale = float(diff.norm() * r.double().norm())
                tol = 1e-9 if fp64 else 1e-5
                assert abs(fd - float(adj[j])) <= tol * scale, (fp64, int(j), fd, float(adj[j]))


def test_cg_step_matches_explicit_G(gravlib, orc):
    """At a tiny size the CG step through the C ABI equals the explicit
    formula with the oracle's G."""
    mesh = (6, 5, 3, 20.0, 20.0, 20.0, 10.0)
    rho_true = np.zeros((3, 5, 6))
    rho_true[1:3, 1:4, 2:5] = 400.0
    G = orc.gmatrix(mesh, DATA_COMPS).reshape(2 * 30, 90)
    clean = (G @ rho_true.reshape(-1)).reshape(2, 5, 6)
    d, w = noisy_data(torch.as_tensor(clean), 0.01, seed=4)
    dn, wn = d.numpy().reshape(-1), np.repeat(w.numpy().reshape(2), 30)
    with Plan(mesh, DATA_COMPS, fp64=True) as plan:
        step = cg_step(plan, d.cuda(), w.cuda())
    g = G.T @ (wn * wn * dn)
    Gg = G @ g
    alpha = (g @ g) / ((wn * Gg) @ (wn * Gg) + step.lam * (g @ g))
    m1 = alpha * g
    assert np.linalg.norm(step.m1.cpu().numpy().reshape(-1) - m1) <= 1e-10 * np.linalg.norm(m1)
    assert step.J1 < step.J0


def test_cg_step_512_fp32_vs_fp64(gravlib):
    """512 x 512 x 64 cubes of 20 m, three boxes, gz + gzz with 1% noise: the
    FP32 step agrees with the FP64 step and lowers the objective."""
    mesh, rho, _ = W.boxes512()
    with Plan(mesh, DATA_COMPS, fp64=True) as p64:
        clean = p64.forward(torch.as_tensor(rho, dtype=torch.float64, device="cuda"))
        d, w = noisy_data(clean.cpu(), 0.01, seed=44)
        s64 = cg_step(p64, d.cuda(), w.cuda())
    with Plan(mesh, DATA_COMPS, fp64=False) as p32:
        s32 = cg_step(p32, d.float().cuda(), w.float().cuda(), lam=s64.lam)
    rel = float((s32.m1.double() - s64.m1).norm() / s64.m1.norm())
    assert rel <= 2e-5, rel
    assert s64.J1 < s64.J0 and s32.J1 < s32.J0


def test_cgls_iterates_match_the_oracle(gravlib, orc):
    """The full inversion loop (damped CGLS with depth weights) through the C
    ABI, FP64: every iterate and objective equals the oracle's CGLS on the
    explicit G."""
    from oracle import inversion as oinv

    mesh = (6, 5, 3, 20.0, 20.0, 20.0, 10.0)
    rng = np.random.default_rng(21)
    rho_true = np.zeros((3, 5, 6))
    rho_true[1:3, 1:4, 2:5] = 400.0
    G = orc.gmatrix(mesh, DATA_COMPS)
    clean = np.einsum("cij,j->ci", G, rho_true.reshape(-1)).reshape(2, 5, 6)
    d, w = noisy_data(torch.as_tensor(clean), 0.01, seed=5)
    wd = w.numpy().reshape(2)
    wm = np.repeat(oinv.depth_weights(mesh), 30)
    A = (wd[:, None, None] * G).reshape(60, 90) / wm[None, :]
    lam = 1e-3 * np.linalg.norm(A, 2) ** 2
    iters = 8
    models, obj = oinv.cgls(G, d.numpy().reshape(2, 30), wd, wm, lam, iters)
    with Plan(mesh, DATA_COMPS, fp64=True) as plan:
        res = cgls(plan, d.cuda(), w.cuda(), lam, iters=iters, keep_models=True)
    for k in range(iters):
        got = res.models[k].cpu().numpy().reshape(-1)
        assert np.linalg.norm(got - models[k]) <= 1e-9 * np.linalg.norm(models[k]), k
    assert np.allclose(res.objectives, obj, rtol=1e-9, atol=0)


def test_cgls_512_fp32_vs_fp64(gravlib):
    """512 x 512 x 64, three boxes, gz + gzz with 1% noise, 8 iterations: the
    FP32 loop follows the FP64 loop and the objective falls every iteration."""
    mesh, rho, _ = W.boxes512()
    with Plan(mesh, DATA_COMPS, fp64=True) as p64:
        clean = p64.forward(torch.as_tensor(rho, dtype=torch.float64, device="cuda"))
        d, w = noisy_data(clean.cpu(), 0.01, seed=45)
        step = cg_step(p64, d.cuda(), w.cuda())
        r64 = cgls(p64, d.cuda(), w.cuda(), step.lam, iters=8)
    with Plan(mesh, DATA_COMPS, fp64=False) as p32:
        r32 = cgls(p32, d.float().cuda(), w.float().cuda(), step.lam, iters=8)
    o64, o32 = np.array(r64.objectives), np.array(r32.objectives)
    assert np.all(np.diff(o64) < 0) and np.all(np.diff(o32) < 0)
    assert np.allclose(o32, o64, rtol=1e-4, atol=0)
    rel = float((r32.m.double() - r64.m).norm() / r64.m.norm())
    assert rel <= 1e-3, rel
