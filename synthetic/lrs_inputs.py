"""Synthetic LRS model parameters (regression matrix, residual law, scales).

The paper fits C, mu, Sigma from tracking data that is not available, so the
tests and the benchmark use seeded stand-ins with the paper's shapes
(Eq. LRS: C has (2h+1) N_Q + 1 rows and N_Q columns):

* C is the identity on the block that multiplies the current predictor
  q^{n*} plus N(0, (c_noise/(2h))**2) entries elsewhere; the bias row is zero.
* mu = 0.
* Sigma = s**2 (A A^T / N_Q + 0.1 I) with A ~ N(0, 1), so it is SPD; s = 1e-5
  makes the per-step residual about 1e-5 of the QoI scale, the size of a
  per-step SGS correction.

With these the predicted q^n stays close to q^{n*} and dQ is a small,
correlated perturbation, which keeps long runs stable.
"""

import numpy as np


def synthetic_lrs(n_qoi, h, seed, c_noise=1.0e-5, s=1.0e-5):
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = (2 * h + 1) * n_qoi + 1
    c = rng.normal(0.0, c_noise / (2.0 * h), size=(rows, n_qoi))
    c[h * n_qoi:(h + 1) * n_qoi, :] = np.eye(n_qoi)
    c[rows - 1, :] = 0.0
    mu = np.zeros(n_qoi)
    a = rng.normal(0.0, 1.0, size=(n_qoi, n_qoi))
    sigma = s * s * (a @ a.T / n_qoi + 0.1 * np.eye(n_qoi))
    return c, mu, sigma
