"""Pins for Philox4x64-10, the Box-Muller normals, the LRS model and KS."""

import math

import numpy as np
import pytest
import scipy.stats

from oracle import philox
from oracle.ks import ks_distance
from oracle.lrs import LRSModel


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((5, 7), (3, 1, 2, 9)), ((2**64 - 1, 12345), (2**63, 0, 7, 1))])
def test_philox_matches_numpy(key, ctr):
    """numpy.random.Philox is the same 4x64-10 generator; it increments the
    counter before each block, so block c is numpy's first block from c - 1."""
    prev = list(ctr)
    # decrement the 256-bit counter
    for i in range(4):
        if prev[i] > 0:
            prev[i] -= 1
            break
        prev[i] = 2**64 - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    want = [int(x) for x in bg.random_raw(4)]
    assert philox.philox4x64_10(ctr, key) == want


def test_own_log_and_trig_accuracy():
    rng = np.random.default_rng(0)
    for x in list(rng.uniform(0, 1, 2000)) + [2.0**-53, 0.5, 1.0, 0.70710678, 1.0 - 2**-53]:
        assert abs(philox.own_log(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))
    for u in list(rng.integers(0, 2**53, 2000) / 2.0**53) + [0.0, 0.25, 0.5, 0.75]:
        c, s = philox.own_cos_sin_2pi(u)
        assert abs(c - math.cos(2 * math.pi * u)) < 1e-15
        assert abs(s - math.sin(2 * math.pi * u)) < 1e-15


def test_normals_statistics():
    z = np.concatenate([philox.normals(99, 0, n, 1, 12) for n in range(4000)])
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 0.03
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3


def test_normals_are_keyed_by_step_member_stream():
    a = philox.normals(1, 0, 5, 1, 4)
    assert a == philox.normals(1, 0, 5, 1, 4)
    assert a != philox.normals(1, 1, 5, 1, 4)
    assert a != philox.normals(1, 0, 6, 1, 4)
    assert a != philox.normals(1, 0, 5, 2, 4)


def test_lrs_history_ordering_and_scaling():
    """A C with one nonzero entry picks out one input: row (k-1) N_Q + j of C
    multiplies q^{n-k}_j / sigma_j; the target is rescaled by sigma_i."""
    nq, h = 3, 4
    sig = np.array([2.0, 3.0, 5.0])
    rows = (2 * h + 1) * nq + 1
    qh = np.arange(h * nq, dtype=float).reshape(h, nq) + 1.0
    qsh = -np.arange(h * nq, dtype=float).reshape(h, nq) - 1.0
    qstar = np.array([0.5, 0.25, 0.125])
    zero = np.zeros((nq, nq))
    for k in range(1, h + 1):
        for j in range(nq):
            c = np.zeros((rows, nq))
            c[(k - 1) * nq + j, 1] = 1.0
            m = LRSModel(c, np.zeros(nq), zero + 1e-300 * np.eye(nq), sig, h, qh, qsh)
            out = m.predict(qstar, np.zeros(nq))
            assert out[1] == pytest.approx(sig[1] * qh[k - 1, j] / sig[j], rel=1e-15)
            c = np.zeros((rows, nq))
            c[(h + 1) * nq + (k - 1) * nq + j, 2] = 1.0
            m = LRSModel(c, np.zeros(nq), zero + 1e-300 * np.eye(nq), sig, h, qh, qsh)
            assert m.predict(qstar, np.zeros(nq))[2] == pytest.approx(sig[2] * qsh[k - 1, j] / sig[j], rel=1e-15)
    # identity on the q^{n*} block and a bias: q^n = q^{n*} + sigma * (bias + mu)
    c = np.zeros((rows, nq))
    c[h * nq:(h + 1) * nq] = np.eye(nq)
    c[-1] = [1.0, 0.0, -1.0]
    mu = np.array([0.0, 2.0, 0.0])
    m = LRSModel(c, mu, 1e-300 * np.eye(nq), sig, h, qh, qsh)
    np.testing.assert_allclose(m.predict(qstar, np.zeros(nq)), qstar + sig * (c[-1] + mu), rtol=1e-15)
    # push: most recent first
    m.push(np.array([9.0, 9.0, 9.0]), np.array([8.0, 8.0, 8.0]))
    assert (m.q_hist[0] == 9).all() and (m.q_hist[1] == qh[0]).all()
    assert (m.qs_hist[0] == 8).all() and (m.qs_hist[1] == qsh[0]).all()


def test_lrs_residual_covariance():
    """eta = mu + L z has covariance Sigma (L L^T = Sigma)."""
    nq = 4
    rng = np.random.default_rng(2)
    a = rng.normal(size=(nq, nq))
    sigma = a @ a.T / nq + 0.1 * np.eye(nq)
    c = np.zeros((nq + 1, nq))
    m = LRSModel(c, np.zeros(nq), sigma, np.ones(nq), 0)
    z = rng.normal(size=(200000, nq))
    eta = np.array([m.predict(np.zeros(nq), zz) for zz in z[:20000]])
    cov = np.cov(eta.T)
    np.testing.assert_allclose(cov, sigma, atol=0.05 * np.max(np.abs(sigma)))


def test_ks_matches_scipy():
    rng = np.random.default_rng(3)
    for n1, n2 in [(50, 70), (300, 300), (1000, 17)]:
        a = rng.normal(size=n1)
        b = rng.normal(0.3, 1.2, size=n2)
        assert ks_distance(a, b) == pytest.approx(scipy.stats.ks_2samp(a, b).statistic, abs=1e-14)


def test_lrs_reference_scale_from_first_prediction():
    nq, h = 3, 2
    rows = (2 * h + 1) * nq + 1
    c = np.zeros((rows, nq))
    c[h * nq:(h + 1) * nq] = np.eye(nq)
    m = LRSModel(c, np.zeros(nq), 1e-300 * np.eye(nq), np.array([0.0, 2.0, -1.0]), h)
    qs = np.array([-4.0, 3.0, 0.0])
    out = m.predict(qs, np.zeros(nq))
    np.testing.assert_array_equal(m.sigma_ref, [4.0, 2.0, 1.0])
    np.testing.assert_allclose(out, qs, rtol=1e-15)
