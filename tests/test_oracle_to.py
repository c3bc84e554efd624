"""Pins for the Tau-orthogonal pieces (Sec. 4, App. A)."""

import numpy as np
import pytest

from oracle import to

CASES = [
    (2, False, (1, 12, 10), [("E", "G", 3), ("Z", "G", 3), ("E", "L", 1), ("Z", "L", 1)], 0),
    (2, False, (1, 8, 8), [("E", "B", 1), ("Z", "B", 1)], 0),
    (2, False, (1, 16, 16), [("E", "F", (0, 2)), ("Z", "F", (0, 2)), ("E", "F", (3, 5)), ("Z", "F", (3, 5))], 0),
    (3, True, (4, 16, 6), [("E", "G", 3), ("Z", "G", 3), ("E", "L", 3), ("Z", "L", 3), ("E", "L", 1), ("Z", "L", 1)], 6),
]


def _setup(dim, walls, shape, qois, nmp):
    nz, ny, nx = shape
    return to.TOSetup(dim, nx, ny, nz, walls, qois, nmp)


def _field(setup, shape, seed, dim):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(3,) + shape) * 0.01
    if dim == 2:
        v[2] = 0
    return v * setup.mask


@pytest.mark.parametrize("dim,walls,shape,qois,nmp", CASES)
def test_sensitivity_is_the_gradient(dim, walls, shape, qois, nmp):
    """E and Z are quadratic and Q^mp linear in v, so the central difference
    (Q(v + e phi) - Q(v - e phi)) / 2e equals <V, phi> up to rounding."""
    st = _setup(dim, walls, shape, qois, nmp)
    v = _field(st, shape, 1, dim)
    phi = _field(st, shape, 2, dim)
    vs = st.sensitivities(v)
    eps = 0.5
    dq = (st.qoi_values(v + eps * phi) - st.qoi_values(v - eps * phi)) / (2 * eps)
    inner = np.array([(vj * phi).sum() for vj in vs])
    np.testing.assert_allclose(dq, inner, rtol=1e-10, atol=1e-18)


@pytest.mark.parametrize("dim,walls,shape,qois,nmp", CASES)
def test_quadratic_expansion_and_self_adjoint_identity(dim, walls, shape, qois, nmp):
    """Q(v + d) = Q(v) + <V, d> + Q(d) for E and Z; Q(v) = <v, V>/2 (E, Z)."""
    st = _setup(dim, walls, shape, qois, nmp)
    v = _field(st, shape, 3, dim)
    d = _field(st, shape, 4, dim)
    q, qd, qvd = st.qoi_values(v), st.qoi_values(d), st.qoi_values(v + d)
    vs = st.sensitivities(v)
    ns = len(qois)
    for i in range(ns):
        assert abs(qvd[i] - (q[i] + (vs[i] * d).sum() + qd[i])) < 1e-12 * abs(qvd[i]) + 1e-20
        assert abs(q[i] - 0.5 * (vs[i] * v).sum()) < 1e-12 * abs(q[i]) + 1e-20
    for i in range(ns, ns + nmp):
        assert abs(qvd[i] - q[i] - qd[i]) < 1e-14


@pytest.mark.parametrize("dim,walls,shape,qois,nmp", CASES)
def test_patterns_orthogonality_and_gamma(dim, walls, shape, qois, nmp):
    """<V_i, O_j> = 0 for i != j, c_ii = 1, <V_i, dv_SGS> = dQ_i, and the
    paper's (c, gamma) route equals dv = sum_k beta_k V_k with beta = G^-1 dQ."""
    st = _setup(dim, walls, shape, qois, nmp)
    v = _field(st, shape, 6, dim)
    vs = st.sensitivities(v)
    g = to.gram(vs)
    assert not to.gram_is_singular(g)
    np.testing.assert_allclose(g, g.T, rtol=1e-14)
    c = to.pattern_coefficients(g)
    np.testing.assert_allclose(np.diag(c), 1.0)
    os_ = to.patterns(c, vs)
    inner = np.array([[(vs[i] * os_[j]).sum() for j in range(st.nq)] for i in range(st.nq)])
    den = to.pattern_norms(c, g)
    off = inner - np.diag(np.diag(inner))
    assert np.max(np.abs(off)) < 1e-9 * np.max(np.abs(np.diag(inner)))
    np.testing.assert_allclose(np.diag(inner), den, rtol=1e-9)
    # closed form: c = diag(G^-1)^-1 G^-1 and den_i = 1/(G^-1)_ii
    gi = np.linalg.inv(g)
    np.testing.assert_allclose(c, gi / np.diag(gi)[:, None], rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(den, 1.0 / np.diag(gi), rtol=1e-8)
    rng = np.random.default_rng(7)
    dq = rng.normal(size=st.nq) * 1e-6
    gamma = dq / den
    dv = to.sgs_increment(gamma, os_)
    np.testing.assert_allclose([(vj * dv).sum() for vj in vs], dq, rtol=1e-8, atol=1e-18)
    beta = np.linalg.solve(g, dq)
    dv2 = np.einsum("k,kazyx->azyx", beta, vs)
    np.testing.assert_allclose(dv, dv2, rtol=1e-7, atol=1e-16)


def test_gram_singular_at_rest_and_detected():
    st = _setup(2, False, (1, 8, 8), [("E", "G", 3), ("Z", "G", 3)], 0)
    vs = st.sensitivities(np.zeros((3, 1, 8, 8)))
    assert to.gram_is_singular(to.gram(vs))
    # duplicated QoI -> rank deficient
    st2 = _setup(2, False, (1, 8, 8), [("E", "G", 3), ("E", "G", 3)], 0)
    v = _field(st2, (1, 8, 8), 1, 2)
    assert to.gram_is_singular(to.gram(st2.sensitivities(v)))


def test_mean_profile_bands():
    """Eq. 3d-mp-band-weights: each band sums to 1 over the fluid rows, is
    symmetric about the channel centre, and peaks at its own wall distance."""
    ny = 40
    w = to.mp_band_weights(ny, 6)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(w, w[:, ::-1], rtol=1e-14, atol=0)
    assert np.all(w[:, 0] == 0) and np.all(w[:, -1] == 0)
    h = 0.5 * (ny - 2)
    centres = np.exp(np.linspace(np.log(0.5), np.log(h), 6))
    dw = np.minimum(np.arange(ny) - 0.5, 2 * h - (np.arange(ny) - 0.5))
    for j in range(6):
        y = int(np.argmax(w[j][: ny // 2]))
        # the peak row is the fluid row whose log wall distance is closest to the centre
        cand = np.arange(1, ny // 2)
        best = cand[np.argmin(np.abs(np.log(dw[cand]) - np.log(centres[j])))]
        assert y == best


def test_mean_profile_band_width_is_the_centre_spacing():
    """Eq. 3d-mp-band-weights (Sec. 7.2): band j is a Gaussian in ln d_w
    centred on ln d_{w,j} with the spacing of the log-spaced centres as its
    width, so w_j(d_{w,j +- 1}) / w_j(d_{w,j}) = exp(-1/2).  ln w_j is then
    exactly quadratic in ln d_w; three rows near the centre give the
    quadratic, whose vertex and curvature are the centre and the width."""
    ny = 2002
    nb = 6
    w = to.mp_band_weights(ny, nb)
    h = 0.5 * (ny - 2)
    centres = np.exp(np.linspace(np.log(0.5), np.log(h), nb))
    spacing = (np.log(h) - np.log(0.5)) / (nb - 1)
    for j in range(nb):
        # three lower-half rows (d_w = y - 1/2) within about one width of the centre
        yc = int(np.clip(round(centres[j] + 0.5), 1, h))
        ys = sorted({max(1, yc - 2 * (j + 1)), yc, min(int(h), yc + 2 * (j + 1))} | {int(h) - 1})[:3]
        if len(ys) < 3:
            ys = [1, 2, 3]
        ld = np.log(np.array(ys) - 0.5)
        lw = np.log(w[j, ys])
        a = np.vstack([np.ones(3), ld, ld * ld]).T
        c0, c1, c2 = np.linalg.solve(a, lw)
        sigma = np.sqrt(-1.0 / (2.0 * c2))
        centre = -c1 / (2.0 * c2)
        assert abs(sigma / spacing - 1.0) < 1e-6, (j, sigma, spacing)
        assert abs(centre - np.log(centres[j])) < 1e-6 * spacing, (j, centre)
        ratio = np.exp(c2 * spacing ** 2)  # w at the next centre over w at this one
        assert abs(ratio - np.exp(-0.5)) < 1e-6
