"""Pins for the velocity sets and the equilibrium (Sec. 2, footnote)."""

import itertools

import numpy as np
import pytest

from oracle import lbm
from oracle.lattice import CS2, Lattice


@pytest.mark.parametrize("dim", [2, 3])
def test_weights_are_the_isotropic_ones(dim):
    """sum w = 1, sum w c_a c_b = c_s^2 delta, 4th moment = c_s^4 (dd + dd + dd):
    these conditions fix the textbook weights uniquely for the given speeds."""
    lat = Lattice(dim)
    c, w = lat.cf[:, :dim], lat.w
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("q,qa,qb->ab", w, c, c), CS2 * np.eye(dim), atol=1e-15)
    m4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    d = np.eye(dim)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(m4, iso, atol=1e-15)
    # odd moments vanish
    np.testing.assert_allclose(np.einsum("q,qa->a", w, c), 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0, atol=1e-15)
    assert lat.q == (9 if dim == 2 else 19)
    for i in range(lat.q):
        assert (lat.c[lat.opp[i]] == -lat.c[i]).all()


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_moments(dim):
    """sum f^eq = rho, sum c f^eq = rho u, sum c c f^eq = rho (c_s^2 I + u u)."""
    lat = Lattice(dim)
    rng = np.random.default_rng(0)
    shape = (2, 3, 4)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, shape)
    u = 0.05 * rng.uniform(-1, 1, (3,) + shape)
    if dim == 2:
        u[2] = 0
    feq = lbm.equilibrium(lat, rho, u)
    r, j = lbm.moments(lat, feq)
    np.testing.assert_allclose(r, rho, rtol=1e-14)
    np.testing.assert_allclose(j, rho * u, atol=1e-15)
    pi = np.einsum("qa,qb,qzyx->abzyx", lat.cf, lat.cf, feq)
    want = rho * (CS2 * np.eye(3)[:, :, None, None, None] + np.einsum("azyx,bzyx->abzyx", u, u))
    if dim == 2:
        want[2, 2] = 0
    np.testing.assert_allclose(pi, want, atol=1e-15)


def test_guo_source_moments():
    """sum_i S_i = 0 and sum_i c_i S_i = (1 - 1/(2 tau)) F."""
    lat = Lattice(3)
    rng = np.random.default_rng(1)
    u = 0.05 * rng.uniform(-1, 1, (3, 2, 3, 4))
    f = 1e-4 * rng.uniform(-1, 1, (3, 2, 3, 4))
    tau = 0.7
    s = lbm.guo_source(lat, f, u, tau)
    np.testing.assert_allclose(s.sum(0), 0, atol=1e-18)
    np.testing.assert_allclose(np.einsum("qa,qzyx->azyx", lat.cf, s), (1 - 0.5 / tau) * f, atol=1e-18)


@pytest.mark.parametrize("dim,walls", [(2, False), (2, True), (3, True)])
def test_stream_is_a_permutation_with_bounce_back(dim, walls):
    """Streaming moves every population exactly once: the multiset of values is
    unchanged; a single tagged population travels along c_i or bounces back."""
    lat = Lattice(dim)
    nz = 1 if dim == 2 else 3
    shape = (lat.q, nz, 6, 5)
    fp = np.arange(np.prod(shape), dtype=np.float64).reshape(shape)
    f = lbm.stream(lat, fp, walls)
    fl = slice(1, 5) if walls else slice(0, 6)
    # fluid outputs are a permutation of fluid inputs
    a = np.sort(f[:, :, fl, :].ravel())
    b = np.sort(fp[:, :, fl, :].ravel())
    np.testing.assert_array_equal(a, b)
    for i, j in itertools.product(range(lat.q), range(1)):
        cx, cy, cz = lat.c[i]
        x, y, z = 2, 2, 0
        assert f[i, (z + cz) % nz, y + cy, (x + cx) % 5] == fp[i, z, y, x]
    if walls:
        i = [k for k in range(lat.q) if tuple(lat.c[k]) == (0, 1, 0)][0]
        assert f[i, 0, 1, 3] == fp[lat.opp[i], 0, 1, 3]
