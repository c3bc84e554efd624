"""Compact convolution filters of Sec. 4.1 as dense kernels, applied literally.

  Gaussian low-pass G_s (Eq. gaussian): exp(-|r|^2/(2 s^2)) over the box
    r in [-alpha s, alpha s]^d, normalised to sum 1 (alpha = 4 in 2-D, 2 in 3-D).
  Laplacian high-pass L_s (Eq. laplace): the biharmonic stencil
    l = [1, -4, 6, -4, 1] placed along each axis through the origin,
    L_1(r) = sum_a l(|r_a| + 2) prod_{b != a} delta(r_b, 0) with 0-based l,
    dilated to scale s by a Kronecker product with the all-ones s^d block and
    normalised so that sum |L_s| = 2.
  Binomial B3: [1, 2, 1]/4 along every axis (the 3x3 pattern filter of the
    64^2 Kolmogorov workload; not one of the paper's filters).

  Sharp Fourier band R_[l,m] (Sec. 4.1, Eq. scale-aware-energy-fourier, App. E):
    keeps the Fourier modes with l - 1/2 <= |k| < m + 1/2, k the integer
    wavenumber vector of a periodic 2-D grid; defined on periodic domains only.

Filters act on the fluid nodes Omega: periodic along x and z; along y with walls
the field is extended by zeros (Sec. 4.1, zero padding) and the output is kept
only on fluid rows, so each filter is a self-adjoint operator on Omega.
"""

import numpy as np

ELL = np.array([1.0, -4.0, 6.0, -4.0, 1.0])


def gaussian_kernel(s, dim):
    alpha = 4 if dim == 2 else 2
    r = int(round(alpha * s))
    ax = np.arange(-r, r + 1, dtype=np.float64)
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    rr = sum(g * g for g in grids)
    k = np.exp(-rr / (2.0 * s * s))
    return k / k.sum()


def laplacian_kernel(s, dim):
    l1 = np.zeros((5,) * dim)
    for idx in np.ndindex(*l1.shape):
        r = [i - 2 for i in idx]
        val = 0.0
        for a in range(dim):
            if all(r[b] == 0 for b in range(dim) if b != a):
                val += ELL[abs(r[a]) + 2]
        l1[idx] = val
    ls = np.kron(l1, np.ones((s,) * dim))
    return ls * (2.0 / np.abs(ls).sum())


def binomial_kernel(dim):
    b = np.array([1.0, 2.0, 1.0]) / 4.0
    k = b
    for _ in range(dim - 1):
        k = np.multiply.outer(k, b)
    return k


def kernel(kind, s, dim):
    if kind == "G":
        return gaussian_kernel(s, dim)
    if kind == "L":
        return laplacian_kernel(s, dim)
    if kind == "B":
        return binomial_kernel(dim)
    raise ValueError(kind)


def shifted(a, r, walls):
    """b(x) = a(x - r) for a field a[..., z, y, x]; r = (rx, ry, rz).
    Periodic along x and z; along y periodic, or zero-filled with walls."""
    rx, ry, rz = r
    b = np.roll(a, shift=(rz, rx), axis=(-3, -1))
    if walls:
        ny = a.shape[-2]
        out = np.zeros_like(b)
        if abs(ry) < ny:
            if ry >= 0:
                out[..., ry:, :] = b[..., :ny - ry, :]
            else:
                out[..., :ny + ry, :] = b[..., -ry:, :]
        return out
    return np.roll(b, ry, axis=-2)


def apply_kernel(a, k, mask, walls):
    """(K * a)(x) = sum_r K(r) a(x - r) on Omega (a is zeroed off Omega first)."""
    dim = k.ndim
    am = a * mask
    out = np.zeros_like(am)
    rad = [(n - 1) // 2 for n in k.shape]
    for idx in zip(*np.nonzero(k)):
        if dim == 2:
            ry, rx = idx[0] - rad[0], idx[1] - rad[1]
            r = (rx, ry, 0)
        else:
            rz, ry, rx = idx[0] - rad[0], idx[1] - rad[1], idx[2] - rad[2]
            r = (rx, ry, rz)
        out += k[idx] * shifted(am, r, walls)
    return out * mask


def fourier_band(a, lo, hi):
    """R_[lo,hi] a on a periodic 2-D field a[..., 1, ny, nx] (Eq. scale-aware-energy-fourier):
    F^-1 (mask F a) with the mask 1 where lo - 1/2 <= |k| < hi + 1/2."""
    ny, nx = a.shape[-2], a.shape[-1]
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    mask = (kk >= lo - 0.5) & (kk < hi + 0.5)
    return np.real(np.fft.ifft2(np.fft.fft2(a, axes=(-2, -1)) * mask, axes=(-2, -1)))
