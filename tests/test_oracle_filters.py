"""Pins for the compact filters (Eqs. gaussian, laplace) and discrete derivatives."""

import numpy as np
import pytest

from oracle import filters, to
from oracle.substrate import central_diff


def test_gaussian_kernel_normalised_and_separable():
    for dim, s, half in [(2, 3, 12), (3, 3, 6), (2, 1, 4), (3, 1, 2)]:
        k = filters.gaussian_kernel(s, dim)
        assert k.shape == (2 * half + 1,) * dim
        assert abs(k.sum() - 1) < 1e-14
        # closed form: product of normalised 1-D Gaussians on [-alpha s, alpha s]
        r = np.arange(-half, half + 1)
        g1 = np.exp(-r * r / (2.0 * s * s))
        g1 /= g1.sum()
        prod = g1
        for _ in range(dim - 1):
            prod = np.multiply.outer(prod, g1)
        np.testing.assert_allclose(k, prod, rtol=1e-13, atol=1e-18)


def test_laplacian_kernel_hand_values():
    """2-D L_1 is the 5x5 cross [1,-4,12,-4,1] (centre 6+6) scaled by 2/32."""
    k = filters.laplacian_kernel(1, 2)
    want = np.zeros((5, 5))
    want[2, :] += [1, -4, 6, -4, 1]
    want[:, 2] += [1, -4, 6, -4, 1]
    np.testing.assert_allclose(k, want * (2.0 / 32.0), rtol=1e-15)
    for dim, s in [(2, 1), (2, 3), (3, 1), (3, 3)]:
        k = filters.laplacian_kernel(s, dim)
        assert k.shape == (5 * s,) * dim
        assert abs(k.sum()) < 1e-14
        assert abs(np.abs(k).sum() - 2.0) < 1e-14
        np.testing.assert_allclose(k, np.flip(k), rtol=0, atol=0)
    # dilation: L_3 in 2-D has 3x3 blocks of equal value; centre block = 12 * scale
    k3 = filters.laplacian_kernel(3, 2)
    c = k3[6:9, 6:9]
    assert np.all(c == c[0, 0]) and c[0, 0] > 0
    assert abs(c[0, 0] / k3[6, 0] - 12.0) < 1e-12  # centre vs outer arm tip value 1


def _shift_zero_y(a, r, walls):
    """b(z, y, x) = a(z - rz, y - ry, x - rx): np.roll along x and z, and along
    y either np.roll (periodic) or a zero-padded slice (walls)."""
    rx, ry, rz = r
    b = np.roll(a, shift=(rz, rx), axis=(0, 2))
    if not walls:
        return np.roll(b, ry, axis=1)
    ny = a.shape[1]
    p = np.pad(b, ((0, 0), (abs(ry), abs(ry)), (0, 0)))
    return p[:, abs(ry) - ry: abs(ry) - ry + ny, :]


@pytest.mark.parametrize("walls", [False, True])
def test_laplacian_l3_is_box_then_strided_cross(walls):
    """Eq. laplace: L_3 is L_1 dilated by the 3^3 block of ones, so it equals
    c C_3 * B_3, the 27-point box followed by the 13-point cross of
    l = [1, -4, 6, -4, 1] at stride 3, with c = 2 / (27 * 48) from sum |L_3| = 2.
    Applied with zero extension beyond the walls, the box must also be taken
    on the solid rows (whose input is zero but whose box is not) for the two
    passes to give the dense kernel's P K P on Omega."""
    rng = np.random.default_rng(5)
    shape = (13, 17, 15)
    mask = np.ones(shape)
    if walls:
        mask[:, 0, :] = 0.0
        mask[:, -1, :] = 0.0
    a = rng.standard_normal(shape) * mask
    dense = filters.apply_kernel(a, filters.laplacian_kernel(3, 3), mask, walls)
    box = sum(_shift_zero_y(a, (dx, dy, dz), walls) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
    cross = 18.0 * box
    for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        for k, w in ((3, -4.0), (6, 1.0)):
            cross = cross + w * (_shift_zero_y(box, tuple(k * c for c in e), walls)
                                 + _shift_zero_y(box, tuple(-k * c for c in e), walls))
    np.testing.assert_allclose(cross * mask / (27.0 * 48.0) * 2.0, dense, rtol=0, atol=1e-13)
    if walls:
        # dropping the solid rows' box changes the rows within 6 of a wall
        cut = _shift_zero_y(box * mask, (0, 0, 0), walls)
        wrong = 18.0 * cut
        for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            for k, w in ((3, -4.0), (6, 1.0)):
                wrong = wrong + w * (_shift_zero_y(cut, tuple(k * c for c in e), walls)
                                     + _shift_zero_y(cut, tuple(-k * c for c in e), walls))
        assert np.abs(wrong * mask / 648.0 - dense).max() > 1e-3


def _mode(shape, kvec):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.cos(kvec[0] * x + kvec[1] * y + kvec[2] * z), (x, y, z)


@pytest.mark.parametrize("kind,s,dim", [("G", 3, 2), ("L", 3, 2), ("L", 1, 2), ("B", 1, 2), ("G", 3, 3), ("L", 3, 3), ("L", 1, 3)])
def test_filter_fourier_symbol(kind, s, dim):
    """On a periodic grid a symmetric kernel maps cos(k.x) to K_hat(k) cos(k.x),
    K_hat(k) = sum_r K(r) cos(k.r) (closed form of a convolution)."""
    shape = (1, 32, 32) if dim == 2 else (16, 16, 16)
    nz, ny, nx = shape
    kvec = (2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny, (2 * np.pi * 1 / nz) if dim == 3 else 0.0)
    f, _ = _mode(shape, kvec)
    k = filters.kernel(kind, s, dim)
    rad = [(n - 1) // 2 for n in k.shape]
    sym = 0.0
    for idx in np.ndindex(*k.shape):
        r = [i - rr for i, rr in zip(idx, rad)]
        if dim == 2:
            kr = kvec[1] * r[0] + kvec[0] * r[1]
        else:
            kr = kvec[2] * r[0] + kvec[1] * r[1] + kvec[0] * r[2]
        sym += k[idx] * np.cos(kr)
    out = filters.apply_kernel(f, k, np.ones(shape), walls=False)
    np.testing.assert_allclose(out, sym * f, atol=1e-13)


@pytest.mark.parametrize("kind,s,dim", [("G", 3, 2), ("L", 3, 2), ("G", 3, 3), ("L", 3, 3), ("L", 1, 3)])
@pytest.mark.parametrize("walls", [False, True])
def test_filter_self_adjoint_on_omega(kind, s, dim, walls):
    """<R a, b> = <a, R b> on Omega, periodic and zero-padded (Sec. 4.1)."""
    rng = np.random.default_rng(3)
    shape = (1, 11, 9) if dim == 2 else (5, 9, 7)
    mask = np.ones(shape)
    if walls:
        mask[:, 0, :] = 0
        mask[:, -1, :] = 0
    a = rng.normal(size=shape) * mask
    b = rng.normal(size=shape) * mask
    k = filters.kernel(kind, s, dim)
    ra = filters.apply_kernel(a, k, mask, walls)
    rb = filters.apply_kernel(b, k, mask, walls)
    assert abs((ra * b).sum() - (a * rb).sum()) < 1e-12 * max(1.0, abs((ra * b).sum()))
    assert np.all(ra[mask == 0] == 0)


def test_zero_padding_matches_brute_force():
    """With walls the filtered value at a fluid node is the kernel sum over fluid
    nodes only (brute force over every offset, periodic in x)."""
    rng = np.random.default_rng(4)
    shape = (1, 8, 6)
    mask = np.ones(shape)
    mask[:, 0, :] = 0
    mask[:, -1, :] = 0
    a = rng.normal(size=shape) * mask
    k = filters.laplacian_kernel(1, 2)
    out = filters.apply_kernel(a, k, mask, walls=True)
    ny, nx = 8, 6
    for y in range(1, ny - 1):
        for x in range(nx):
            acc = 0.0
            for ry in range(-2, 3):
                for rx in range(-2, 3):
                    yy = y - ry
                    if 1 <= yy <= ny - 2:
                        acc += k[ry + 2, rx + 2] * a[0, yy, (x - rx) % nx]
            assert abs(out[0, y, x] - acc) < 1e-14


def test_central_difference_of_a_mode():
    """D sin(k x) = sin(k) cos(k x) exactly for the central difference."""
    nx = 16
    x = np.arange(nx)
    k = 2 * np.pi * 3 / nx
    u = np.sin(k * x)[None, None, :] * np.ones((2, 3, 1))
    d = central_diff(u, 0, walls=False)
    np.testing.assert_allclose(d, np.sin(k) * np.cos(k * x)[None, None, :] * np.ones((2, 3, 1)), atol=1e-15)


@pytest.mark.parametrize("dim,walls", [(2, False), (2, True), (3, False), (3, True)])
def test_curl_adjoint(dim, walls):
    """<curl a, b> = <a, curl* b> on Omega (App. A, vanishing boundary terms)."""
    rng = np.random.default_rng(5)
    shape = (1, 9, 8) if dim == 2 else (5, 7, 6)
    mask = np.ones(shape)
    if walls:
        mask[:, 0, :] = 0
        mask[:, -1, :] = 0
    a = rng.normal(size=(3,) + shape) * mask
    if dim == 2:
        a[2] = 0
    nb = 1 if dim == 2 else 3
    b = rng.normal(size=(nb,) + shape) * mask
    ca = to.curl(a, dim, walls) * mask
    cb = to.curl_adjoint(b, dim, walls) * mask
    assert abs((ca * b).sum() - (a * cb).sum()) < 1e-12


def test_fourier_bands_are_orthogonal_projections():
    """R_[l,m] is idempotent and self-adjoint, bands covering the spectrum sum
    to the identity, and band energies add up to the total (Parseval)."""
    rng = np.random.default_rng(9)
    a = rng.normal(size=(2, 1, 32, 32))
    bands = [(0, 3), (4, 9), (10, 40)]
    parts = [filters.fourier_band(a, lo, hi) for lo, hi in bands]
    np.testing.assert_allclose(sum(parts), a, atol=1e-12)
    for (lo, hi), r in zip(bands, parts):
        np.testing.assert_allclose(filters.fourier_band(r, lo, hi), r, atol=1e-12)
    b = rng.normal(size=a.shape)
    rb = filters.fourier_band(b, 4, 9)
    assert abs((parts[1] * b).sum() - (a * rb).sum()) < 1e-10
    e_tot = 0.5 * (a * a).sum()
    assert abs(sum(0.5 * (r * r).sum() for r in parts) - e_tot) < 1e-10 * e_tot
    # a single mode lands in the band of its wavenumber |k| = 5
    y, x = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    mode = np.cos(2 * np.pi * (3 * x + 4 * y) / 32)[None, None]
    np.testing.assert_allclose(filters.fourier_band(mode, 4, 9), mode, atol=1e-12)
    np.testing.assert_allclose(filters.fourier_band(mode, 0, 3), 0, atol=1e-12)
