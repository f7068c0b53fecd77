"""Oracle of the inversion loop: damped CGLS on the explicit kernel matrix.

Test infrastructure, not product code (see the package header).

The paper's motivation for a fast forward is least-squares density inversion
(Sec. 1, Sec. 4); it prints no inversion algorithm.  The problem solved here
is the Tikhonov one with data and depth weights,

    min_m  ||W_d (G m - d)||^2 + lam ||W_m m||^2,

W_d = diag(1 / sigma_c) per component and W_m = diag(w_n) per layer, with the
depth weights of Li and Oldenburg (1996), w_n = (h + (n + 1/2) dz)^(-beta/2)
(depth of the layer centre below the stations; beta = 2 undoes the 1/z^2
decay of the gravity kernel), scaled to a largest value of 1.  In the
variable x = W_m m it is the damped least-squares problem
min ||A x - b||^2 + lam ||x||^2 with A = W_d G W_m^-1, b = W_d d, solved by
conjugate gradients on the normal equations (CGLS: Hestenes and Stiefel
1952; Bjorck 1996, the damped form), written out here with numpy on the
dense A.  Each step is the textbook recurrence, in that order:

    x0 = 0, r0 = b, s0 = A^T r0, p0 = s0, gamma0 = ||s0||^2
    q = A p;  alpha = gamma / (||q||^2 + lam ||p||^2)
    x += alpha p;  r -= alpha q;  s = A^T r - lam x
    gamma' = ||s||^2;  p = s + (gamma' / gamma) p
"""
from __future__ import annotations

import numpy as np


def depth_weights(mesh, beta: float = 2.0) -> np.ndarray:
    """w_n = (h + (n + 1/2) dz)^(-beta/2), n < nz, scaled so max w_n = 1."""
    nz, dz, h = int(mesh[2]), float(mesh[5]), float(mesh[6])
    z = h + (np.arange(nz) + 0.5) * dz
    w = z ** (-beta / 2.0)
    return w / w.max()


def cgls(G: np.ndarray, d: np.ndarray, wd: np.ndarray, wm_cells: np.ndarray, lam: float, iters: int):
    """Damped CGLS in the weighted variables.

    G: [nc][nd][nm] (oracle.gmatrix); d: [nc][nd]; wd: [nc] data weights;
    wm_cells: [nm] model weight of every cell (w_n of its layer).
    Returns (models, objectives): the model m_k = W_m^-1 x_k after each of
    the `iters` steps ([iters][nm]) and J(m_k) = ||W_d (G m_k - d)||^2 +
    lam ||W_m m_k||^2 for k = 0 .. iters ([iters + 1])."""
    nc, nd, nm = G.shape
    A = (wd[:, None, None] * G).reshape(nc * nd, nm) / wm_cells[None, :]
    b = (wd[:, None] * d).reshape(nc * nd)

    def objective(x):
        res = A @ x - b
        return float(res @ res + lam * (x @ x))

    x = np.zeros(nm)
    r = b.copy()
    s = A.T @ r
    p = s.copy()
    gamma = float(s @ s)
    models, objectives = [], [objective(x)]
    for _ in range(iters):
        if gamma == 0.0:  # converged exactly: the iterate stays
            models.append(x / wm_cells)
            objectives.append(objective(x))
            continue
        q = A @ p
        alpha = gamma / (float(q @ q) + lam * float(p @ p))
        x = x + alpha * p
        r = r - alpha * q
        s = A.T @ r - lam * x
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        models.append(x / wm_cells)
        objectives.append(objective(x))
    return np.array(models), np.array(objectives)
