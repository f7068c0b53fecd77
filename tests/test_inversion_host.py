"""The inversion driver's host logic on the CPU: `cgls`, `depth_weights` and
`noisy_data` of the package, driven through an operator made of the oracle's
explicit G applied as a dense matrix (no device), against the oracle's CGLS.
The GPU test of the same loop runs the operator through the C ABI."""
import numpy as np
import torch

import oracle
from oracle import inversion as oinv
from paper_2005_10160_gb300.inversion import cgls, depth_weights, noisy_data

MESH = (6, 5, 3, 20.0, 20.0, 20.0, 10.0)
COMPS = 0x41  # gz + gzz


class ExplicitPlan:
    """The plan interface the loop uses (mesh, forward, adjoint) with the
    oracle's G [nc][nd][nm] as a dense matrix."""

    def __init__(self, mesh, G):
        self.mesh, self.G = mesh, torch.as_tensor(G)

    def forward(self, rho):
        nx, ny = self.mesh[:2]
        return torch.einsum("cij,j->ci", self.G, rho.reshape(-1)).reshape(-1, ny, nx)

    def adjoint(self, r):
        nx, ny, nz = self.mesh[:3]
        return torch.einsum("cij,ci->j", self.G, r.reshape(self.G.shape[0], -1)).reshape(nz, ny, nx)


def test_cgls_driver_follows_the_oracle_recurrence():
    """Every iterate and objective of the package's loop equals the oracle's
    CGLS on the same explicit G (FP64; the two differ only in rounding order,
    which CG amplifies to about 1e-12 after 8 iterations)."""
    oracle.build()
    G = oracle.gmatrix(MESH, COMPS)
    rho_true = np.zeros((3, 5, 6))
    rho_true[1:3, 1:4, 2:5] = 400.0
    clean = np.einsum("cij,j->ci", G, rho_true.reshape(-1)).reshape(2, 5, 6)
    d, w = noisy_data(torch.as_tensor(clean), 0.01, seed=5)
    wd = w.numpy().reshape(2)
    wm = np.repeat(oinv.depth_weights(MESH), 30)
    A = (wd[:, None, None] * G).reshape(60, 90) / wm[None, :]
    lam = 1e-3 * np.linalg.norm(A, 2) ** 2
    iters = 8
    models, obj = oinv.cgls(G, d.numpy().reshape(2, 30), wd, wm, lam, iters)
    res = cgls(ExplicitPlan(MESH, G), d, w, lam, iters=iters, keep_models=True)
    for k in range(iters):
        got = res.models[k].numpy().reshape(-1)
        assert np.linalg.norm(got - models[k]) <= 1e-10 * np.linalg.norm(models[k]), k
    assert np.allclose(res.objectives, obj, rtol=1e-10, atol=0)
    assert np.isnan(res.ms_per_iteration)  # timed with CUDA events only on a GPU


def test_depth_weights_shape_and_scale():
    """One weight per layer, broadcastable over [nz][ny][nx], largest 1 at
    the top layer and in the ratio of (h + (n + 1/2) dz)^(-beta/2)."""
    w = depth_weights(MESH, beta=2.0, dtype=torch.float64)
    assert tuple(w.shape) == (3, 1, 1)
    z = MESH[6] + (np.arange(3) + 0.5) * MESH[5]
    assert np.allclose(w.reshape(-1).numpy(), z[0] / z, rtol=1e-15)


def test_noisy_data_noise_level_and_weights():
    """The added noise has the requested RMS per component (to sampling
    error), the weights are 1 / sigma_c, and the same seed gives the same data."""
    rng = np.random.default_rng(3)
    clean = torch.as_tensor(rng.normal(size=(2, 64, 64)) * np.array([1.0, 1e-3])[:, None, None])
    d, w = noisy_data(clean, 0.05, seed=9)
    rms = clean.pow(2).mean(dim=(1, 2)).sqrt()
    noise_rms = (d - clean).pow(2).mean(dim=(1, 2)).sqrt()
    assert torch.allclose(noise_rms / rms, torch.full((2,), 0.05, dtype=torch.float64), rtol=0.05)
    assert torch.allclose(w.reshape(-1), 1.0 / (0.05 * rms))
    d2, _ = noisy_data(clean, 0.05, seed=9)
    assert torch.equal(d, d2)
