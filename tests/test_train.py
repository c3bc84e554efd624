"""LRS training (Sec. 4.4): the oracle's literal fit recovers a known model,
satisfies the ridge normal equations, and the library's fit equals it."""

import numpy as np

from oracle import train as otrain
from paper_2609_32892_b300 import train as ptrain


def _series(c_true, mu, sigma, h, t, seed, sref):
    """Series generated by an LRS model: q^{n*} is a noisy function of the past,
    q^n = LRS(q_h)."""
    rng = np.random.default_rng(seed)
    nq = len(mu)
    q = np.zeros((t, nq))
    qs = np.zeros((t, nq))
    lch = np.linalg.cholesky(sigma)
    q[:h] = sref * (1 + 0.1 * rng.normal(size=(h, nq)))
    qs[:h] = q[:h]
    for n in range(h, t):
        qs[n] = q[n - 1] + 0.05 * sref * rng.normal(size=nq)
        x = np.concatenate([q[n - k] / sref for k in range(1, h + 1)] + [qs[n] / sref] +
                           [qs[n - k] / sref for k in range(1, h + 1)] + [[1.0]])
        q[n] = sref * (x @ c_true + mu + lch @ rng.normal(size=nq))
    return q, qs


def _truth(nq, h, seed):
    rng = np.random.default_rng(seed)
    rows = (2 * h + 1) * nq + 1
    c = 0.02 * rng.normal(size=(rows, nq))
    c[h * nq:(h + 1) * nq] += 0.9 * np.eye(nq)
    c[-1] = 0.05
    a = rng.normal(size=(nq, nq))
    return c, np.array([0.01, -0.02, 0.0]), 1e-3 * (a @ a.T / nq + 0.2 * np.eye(nq))


def test_oracle_fit_recovers_a_known_model():
    nq, h = 3, 2
    sref = np.array([2.0, 0.5, 3.0])
    c, mu, sig = _truth(nq, h, 1)
    q, qs = _series(c, mu, sig, h, 6000, 2, sref)
    cf, muf, sigf, lams = otrain.fit(q, qs, h, sref, 0.0)
    assert np.all(lams == 0)
    # the residual law is recovered (C and mu trade off along the bias direction)
    np.testing.assert_allclose(sigf, sig, rtol=0.1, atol=2e-5)
    np.testing.assert_allclose(cf[h * nq:(h + 1) * nq], c[h * nq:(h + 1) * nq], atol=0.05)


def test_ridge_normal_equations_and_penalties():
    rng = np.random.default_rng(3)
    nq, h, t = 3, 3, 400
    q = rng.normal(size=(t, nq)) + 5
    qs = q + 0.1 * rng.normal(size=(t, nq))
    sref = np.array([1.0, 2.0, 0.5])
    lam = 0.7
    c, mu, sig, lams = otrain.fit(q, qs, h, sref, lam)
    qh, tq = otrain.design(q, qs, h, sref)
    corr = (q[h:] - qs[h:]) / sref
    np.testing.assert_allclose(lams, lam * (corr.std(axis=0) / corr.std(axis=0)[0]) ** 2, rtol=1e-12)
    for i in range(nq):
        grad = qh.T @ (qh @ c[:, i] - tq[:, i]) + lams[i] * c[:, i]
        assert np.max(np.abs(grad)) < 1e-8 * np.max(np.abs(qh.T @ tq[:, i]))
    np.testing.assert_allclose(mu, (tq - qh @ c).mean(axis=0), atol=1e-14)


def test_library_fit_equals_oracle_fit():
    rng = np.random.default_rng(4)
    nq, h, t = 4, 5, 800
    q = rng.normal(size=(t, nq)) * [1, 2, 3, 4] + 10
    qs = q + 0.2 * rng.normal(size=(t, nq))
    sref = np.array([1.0, 2.0, 3.0, 4.0])
    for lam in (0.0, 1.0, 5.0):
        a = otrain.fit(q, qs, h, sref, lam)
        b = ptrain.fit_lrs(q, qs, h, sref, lam)
        for x, y in zip(a, b):
            np.testing.assert_allclose(y, x, rtol=1e-7, atol=1e-10)
