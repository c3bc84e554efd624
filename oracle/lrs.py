"""Linear regression with stochastic residuals (Eq. LRS, Sec. 4.4).

  q^n = LRS(q_h) = q_h C + eta,  eta ~ N(mu, Sigma),
  q_h = [q^{n-1}, ..., q^{n-h}, q^{n*}, q^{n-1*}, ..., q^{n-h*}, 1],
with inputs and targets divided by the reference standard deviations sigma_ref
(no centring; the bias entry is not scaled) and eta living in scaled units.
eta = mu + L z with L the Cholesky factor of Sigma and z standard normals.
The corrected q^n and the predictor q^{n*} are pushed into the histories.

A reference scale given as <= 0 is taken from the first prediction: it becomes
|q^{n*}_i| (1 if that is 0).  The paper scales by the reference trajectories'
standard deviation, which a server admitting new runs does not have; this
reading needs zero initial histories.
"""

import numpy as np


class LRSModel:
    def __init__(self, c, mu, sigma, sigma_ref, h, q_hist=None, qs_hist=None):
        self.c = np.asarray(c, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.l = np.linalg.cholesky(np.asarray(sigma, dtype=np.float64))
        self.sigma_ref = np.asarray(sigma_ref, dtype=np.float64)
        self.h = h
        nq = len(self.mu)
        self.nq = nq
        assert self.c.shape == ((2 * h + 1) * nq + 1, nq)
        # row k holds q^{n-1-k} (most recent first)
        self.q_hist = np.zeros((h, nq)) if q_hist is None else np.array(q_hist, dtype=np.float64)
        self.qs_hist = np.zeros((h, nq)) if qs_hist is None else np.array(qs_hist, dtype=np.float64)

    def inputs(self, qstar):
        s = self.sigma_ref
        return np.concatenate([(self.q_hist / s).ravel(), qstar / s, (self.qs_hist / s).ravel(), [1.0]])

    def predict(self, qstar, z):
        auto = self.sigma_ref <= 0.0
        if np.any(auto):
            a = np.abs(qstar)
            self.sigma_ref = np.where(auto, np.where(a > 0.0, a, 1.0), self.sigma_ref)
        x = self.inputs(qstar)
        qhat = x @ self.c + self.mu + self.l @ np.asarray(z)
        return self.sigma_ref * qhat

    def push(self, q, qstar):
        if self.h == 0:
            return
        self.q_hist = np.vstack([q[None], self.q_hist[:-1]])
        self.qs_hist = np.vstack([qstar[None], self.qs_hist[:-1]])
