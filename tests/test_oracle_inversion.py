"""Pins of the inversion oracle (damped CGLS with depth weights on the
explicit G), against the mathematics rather than against itself: CG on the
normal equations reaches the exact minimiser of the quadratic (in exact
arithmetic within as many steps as there are unknowns; in floating point a
few more), never increases the objective, and its first step is the exact
line search along the steepest-descent direction."""
import numpy as np
import pytest

import oracle
from oracle import inversion as oinv

MESH = (3, 2, 2, 10.0, 12.0, 8.0, 2.0)  # 12 unknowns
COMPS = 0x41                              # gz + gzz: 12 data


@pytest.fixture(scope="module")
def problem():
    oracle.build()
    G = oracle.gmatrix(MESH, COMPS)
    rng = np.random.default_rng(11)
    m_true = rng.uniform(-300, 300, G.shape[2])
    d = np.einsum("cij,j->ci", G, m_true)
    wd = 1.0 / (0.01 * np.sqrt((d ** 2).mean(axis=1)))
    wm = np.repeat(oinv.depth_weights(MESH), MESH[0] * MESH[1])
    A = (wd[:, None, None] * G).reshape(-1, G.shape[2]) / wm[None, :]
    lam = 1e-3 * np.linalg.norm(A, 2) ** 2
    return G, d, wd, wm, A, lam


def test_depth_weights_undo_the_depth_decay():
    w = oinv.depth_weights(MESH, beta=2.0)
    z = MESH[6] + (np.arange(MESH[2]) + 0.5) * MESH[5]
    assert w.max() == 1.0 and np.all(np.diff(w) < 0)
    assert np.allclose(w * z, (w * z)[0], rtol=1e-14)  # beta = 2: w ~ 1/z
    w3 = oinv.depth_weights(MESH, beta=3.0)
    assert np.allclose(w3 * z ** 1.5, (w3 * z ** 1.5)[0], rtol=1e-14)


def test_cgls_reaches_the_direct_solution(problem):
    G, d, wd, wm, A, lam = problem
    b = (wd[:, None] * d).reshape(-1)
    x_star = np.linalg.solve(A.T @ A + lam * np.eye(A.shape[1]), A.T @ b)
    models, obj = oinv.cgls(G, d, wd, wm, lam, iters=2 * A.shape[1])
    x_k = models[-1] * wm
    assert np.linalg.norm(x_k - x_star) <= 1e-10 * np.linalg.norm(x_star)
    J_star = float(np.sum((A @ x_star - b) ** 2) + lam * x_star @ x_star)
    assert abs(obj[-1] - J_star) <= 1e-8 * J_star


def test_cgls_objective_never_increases(problem):
    G, d, wd, wm, A, lam = problem
    _, obj = oinv.cgls(G, d, wd, wm, lam, iters=10)
    assert np.all(np.diff(obj) <= 1e-12 * obj[0])
    assert obj[-1] < 0.5 * obj[0]


def test_first_step_is_the_exact_line_search(problem):
    G, d, wd, wm, A, lam = problem
    b = (wd[:, None] * d).reshape(-1)
    g = A.T @ b
    alpha = (g @ g) / (np.sum((A @ g) ** 2) + lam * (g @ g))
    models, _ = oinv.cgls(G, d, wd, wm, lam, iters=1)
    assert np.allclose(models[0] * wm, alpha * g, rtol=1e-12, atol=0)


def test_pins_catch_a_sign_slip_in_the_damping(problem):
    """A plausible mistake (adding instead of subtracting lam x in the
    residual of the normal equations) breaks the direct-solution pin."""
    G, d, wd, wm, A, lam = problem
    b = (wd[:, None] * d).reshape(-1)
    x_star = np.linalg.solve(A.T @ A + lam * np.eye(A.shape[1]), A.T @ b)
    x = np.zeros(A.shape[1])
    r = b.copy()
    s = A.T @ r
    p = s.copy()
    gamma = s @ s
    for _ in range(2 * A.shape[1]):
        q = A @ p
        alpha = gamma / (q @ q + lam * (p @ p))
        x = x + alpha * p
        r = r - alpha * q
        s = A.T @ r + lam * x  # the slip
        gamma_new = s @ s
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    assert np.linalg.norm(x - x_star) > 1e-3 * np.linalg.norm(x_star)
