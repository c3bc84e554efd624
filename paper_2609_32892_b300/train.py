"""Fit the LRS time-series model of the TO closure from a tracking run.

Inputs are the corrected QoIs q^n and predictor QoIs q^{n*} of every step of a
tracking run (lbm_qoi rows: q^{n*} and dQ, q^n = q^{n*} + dQ), the history
length h, the reference scales sigma_ref and the base penalty lambda.  The
inputs and targets are divided by sigma_ref (no centring, bias unscaled); each
QoI column i of C gets the penalty lambda_i = lambda (s_i/s_1)^2 with s_i the
standard deviation of the scaled corrections; (mu, Sigma) are the mean and
covariance of the training residuals.  The result feeds lbm_set_lrs.

All columns share one Gram matrix G = Q_h^T Q_h: after its eigendecomposition
G = U diag(e) U^T every column costs two matrix-vector products,
C_i = U diag(1/(e + lambda_i)) U^T Q_h^T Q_i.  Host FP64 (numpy).
"""

import numpy as np


def history_matrix(q, qs, h, sigma_ref):
    """Q_h rows [q^{n-1..n-h}, q^{n*}, q^{n-1*..n-h*}] / sigma, 1 and targets q^n / sigma."""
    q = np.asarray(q, dtype=np.float64) / sigma_ref
    qs = np.asarray(qs, dtype=np.float64) / sigma_ref
    t, nq = q.shape
    rows = t - h
    x = np.empty((rows, (2 * h + 1) * nq + 1))
    for k in range(1, h + 1):
        x[:, (k - 1) * nq:k * nq] = q[h - k:t - k]
        x[:, (h + 1 + k - 1) * nq:(h + 1 + k) * nq] = qs[h - k:t - k]
    x[:, h * nq:(h + 1) * nq] = qs[h:]
    x[:, -1] = 1.0
    return x, q[h:]


def fit_lrs(q, qs, h, sigma_ref, lam):
    sigma_ref = np.asarray(sigma_ref, dtype=np.float64)
    x, y = history_matrix(q, qs, h, sigma_ref)
    corr_sd = (y - x[:, h * len(sigma_ref):(h + 1) * len(sigma_ref)]).std(axis=0)
    lams = lam * (corr_sd / corr_sd[0]) ** 2
    g = x.T @ x
    e, u = np.linalg.eigh(g)
    rhs = u.T @ (x.T @ y)
    c = np.empty((x.shape[1], y.shape[1]))
    for i, li in enumerate(lams):
        c[:, i] = u @ (rhs[:, i] / (e + li))
    res = y - x @ c
    mu = res.mean(axis=0)
    d = res - mu
    sigma = d.T @ d / (len(res) - 1)
    return c, mu, sigma, lams


def series_from_rows(rows, nq):
    """(q^n, q^{n*}) from lbm_qoi rows [step, q*, dQ, gamma, flags]."""
    qs = rows[:, 1:1 + nq]
    return qs + rows[:, 1 + nq:1 + 2 * nq], qs
