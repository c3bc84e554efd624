"""Fitting the LRS model from a tracking run (Sec. 4.4, Eq. LRS and the ridge
problem that follows it), literally.

Training data: for each step n of a tracking run, the corrected QoIs q^n and
the predictor QoIs q^{n*}.  Every row with a full history (n >= h) gives
  input  q_h^n = [q^{n-1}, ..., q^{n-h}, q^{n*}, q^{n-1*}, ..., q^{n-h*}] / sigma_ref, then 1
  target q^n / sigma_ref
(scaled by the reference standard deviations, no mean removal, bias unscaled).
C minimises 1/2 |Q_h X - Q|_F^2 + lambda/2 |X|_F^2, column i with its own
penalty lambda_i = lambda (s_i / s_1)^2, s_i the standard deviation of the
scaled corrections (q^n_i - q^{n*}_i)/sigma_i (the paper's footnote).  The
residual law N(mu, Sigma) is the sample mean and covariance of Q - Q_h C.
"""

import numpy as np


def design(q, qs, h, sigma_ref):
    """Q_h and Q from series q[T][N], qs[T][N] (rows n = h..T-1)."""
    q = np.asarray(q, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64)
    s = np.asarray(sigma_ref, dtype=np.float64)
    rows, targets = [], []
    for n in range(h, len(q)):
        past = [q[n - k] / s for k in range(1, h + 1)]
        past_s = [qs[n - k] / s for k in range(1, h + 1)]
        rows.append(np.concatenate(past + [qs[n] / s] + past_s + [[1.0]]))
        targets.append(q[n] / s)
    return np.array(rows), np.array(targets)


def penalties(q, qs, h, sigma_ref, lam):
    """lambda_i = lambda (s_i / s_1)^2 over the training rows."""
    s = np.asarray(sigma_ref, dtype=np.float64)
    corr = (np.asarray(q)[h:] - np.asarray(qs)[h:]) / s
    sd = corr.std(axis=0)
    return lam * (sd / sd[0]) ** 2


def fit(q, qs, h, sigma_ref, lam):
    """(C, mu, Sigma, lambda_i) of the LRS model."""
    qh, tq = design(q, qs, h, sigma_ref)
    lams = penalties(q, qs, h, sigma_ref, lam)
    m = qh.shape[1]
    c = np.zeros((m, tq.shape[1]))
    for i in range(tq.shape[1]):
        c[:, i] = np.linalg.solve(qh.T @ qh + lams[i] * np.eye(m), qh.T @ tq[:, i])
    res = tq - qh @ c
    return c, res.mean(axis=0), np.cov(res.T).reshape(tq.shape[1], tq.shape[1]), lams


def summed_ks(samples_a, samples_b):
    """Sum over QoIs of the KS distance between long-term distributions (Eq. KS)."""
    from .ks import ks_distance

    return sum(ks_distance(samples_a[:, i], samples_b[:, i]) for i in range(samples_a.shape[1]))
