"""Eddy-viscosity substrates folded into an effective relaxation time (Sec. 5).

tau_eff = (nu + nu_t)/c_s^2 + 1/2 (Eq. eff-relaxation), i.e. tau_eff = tau + 3 nu_t.
"""

import numpy as np

from .lattice import CS2


def smagorinsky_tau_eff(lat, f, feq, rho, tau, c_smag):
    """Smagorinsky from the non-equilibrium stress (Sec. 5.1):
    Pi^neq_ab = sum_i c_ia c_ib (f_i - f_i^eq), |Pi| = sqrt(2 Pi:Pi),
    tau_eff = (tau + sqrt(tau^2 + 18 C^2 |Pi| / rho)) / 2."""
    fneq = f - feq
    pi = np.einsum("qa,qb,qzyx->abzyx", lat.cf, lat.cf, fneq)
    pinorm = np.sqrt(2.0 * (pi * pi).sum(axis=(0, 1)))
    return 0.5 * (tau + np.sqrt(tau * tau + 18.0 * c_smag * c_smag * pinorm / rho))


def central_diff(u, axis, walls):
    """Second-order central difference d/dx_axis in lattice units; periodic in x
    and z; along y with walls the field is zero outside the fluid rows.  The
    input must already be zero on solid rows.  axis: 0 = x, 1 = y, 2 = z."""
    ax = {0: -1, 1: -2, 2: -3}[axis]
    if axis == 1 and walls:
        up = np.zeros_like(u)
        dn = np.zeros_like(u)
        up[..., :-1, :] = u[..., 1:, :]   # u(y+1)
        dn[..., 1:, :] = u[..., :-1, :]   # u(y-1)
        d = 0.5 * (up - dn)
        d[..., 0, :] = 0.0
        d[..., -1, :] = 0.0
        return d
    return 0.5 * (np.roll(u, -1, axis=ax) - np.roll(u, 1, axis=ax))


def wale_tau_eff(v, mask, tau, c_w, dim, walls):
    """WALE (Sec. 5.2): g_ij = d_j v_i by central differences,
    S = (g + g^T)/2, S^d = (g g + (g g)^T)/2 - (1/3) delta tr(g g),
    nu_t = C_w^2 (S^d:S^d)^{3/2} / ((S:S)^{5/2} + (S^d:S^d)^{5/4}), with
    nu_t = 0 where that denominator is below 1e-30 (v locally uniform).
    2-D flows are treated as 3-D flows with d/dz = 0 and v_z = 0."""
    vm = v * mask[None]
    g = np.zeros((3, 3) + mask.shape)
    for i in range(3):
        for j in range(dim):
            g[i, j] = central_diff(vm[i], j, walls)
    s = 0.5 * (g + g.transpose(1, 0, 2, 3, 4))
    g2 = np.einsum("ikzyx,kjzyx->ijzyx", g, g)
    tr = np.einsum("iizyx->zyx", g2)
    sd = 0.5 * (g2 + g2.transpose(1, 0, 2, 3, 4))
    for i in range(3):
        sd[i, i] -= tr / 3.0
    ss = (s * s).sum(axis=(0, 1))
    sdsd = (sd * sd).sum(axis=(0, 1))
    den = ss ** 2.5 + sdsd ** 1.25
    with np.errstate(divide="ignore", invalid="ignore"):
        nut = np.where(den < 1e-30, 0.0, c_w * c_w * sdsd ** 1.5 / np.where(den < 1e-30, 1.0, den))
    return tau + nut / CS2
