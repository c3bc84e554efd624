"""Lattice-Boltzmann building blocks in float64 (Sec. 2; Eqs. LES-1..3).

Array layout: populations f[q, z, y, x]; velocities u[a, z, y, x] with a = x, y, z
(2-D runs have nz = 1 and u_z = 0); scalars rho[z, y, x].
"""

import numpy as np

from .lattice import CS2


def equilibrium(lat, rho, u):
    """Second-order equilibrium of the footnote to Sec. 2:
    f_i^eq = w_i rho (1 + u.c_i/c_s^2 + (u.c_i)^2/(2 c_s^4) - u.u/(2 c_s^2))."""
    cu = np.einsum("qa,azyx->qzyx", lat.cf, u)
    uu = (u * u).sum(axis=0)
    w = lat.w[:, None, None, None]
    return w * rho[None] * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu[None] / (2.0 * CS2))


def moments(lat, f):
    """Mass and momentum, rho = sum_i f_i and rho u = sum_i f_i c_i (Sec. 2)."""
    rho = f.sum(axis=0)
    j = np.einsum("qa,qzyx->azyx", lat.cf, f)
    return rho, j


def relax(f, feq, tau):
    """BGK relaxation, f^a = (1 - dt/tau) f + (dt/tau) f^eq (Eq. LES-1, dt = 1);
    tau may be a per-node field (eddy-viscosity substrate, Eq. eff-relaxation)."""
    return (1.0 - 1.0 / tau) * f + feq / tau


def edm_forcing(lat, fa, rho, u, du):
    """Exact-difference forcing, f^p = f^a + f^eq(rho, u + du) - f^eq(rho, u)
    (Eq. collide-and-stream; Eq. LES-2 with du = du_F + dv_SGS)."""
    return fa + equilibrium(lat, rho, u + du) - equilibrium(lat, rho, u)


def guo_source(lat, force, u, tau):
    """Guo forcing term S_i = (1 - 1/(2 tau)) w_i [(c_i - u)/c_s^2 + (c_i.u) c_i/c_s^4] . F.

    The paper forces with the exact-difference method; Guo's scheme is the
    variant the benchmark configuration names, provided behind a flag.
    """
    q = lat.q
    out = np.empty((q,) + force.shape[1:])
    cu = np.einsum("qa,azyx->qzyx", lat.cf, u)
    for i in range(q):
        ci = lat.cf[i][:, None, None, None]
        term = (ci - u) / CS2 + cu[i][None] * ci / (CS2 * CS2)
        out[i] = lat.w[i] * (term * force).sum(axis=0)
    return (1.0 - 1.0 / (2.0 * tau)) * out


def stream(lat, fp, walls):
    """Pull streaming f_i(x, t+1) = f^p_i(x - c_i, t) (Eq. LES-3), periodic in x
    and z; with walls, halfway bounce-back at the solid rows y = 0 and y = ny-1:
    when x - c_i is solid, f_i(x, t+1) = f^p_{opp(i)}(x, t).  Solid rows keep
    their values (they are never collided)."""
    f = np.empty_like(fp)
    ny = fp.shape[2]
    for i in range(lat.q):
        cx, cy, cz = (int(v) for v in lat.c[i])
        f[i] = np.roll(fp[i], shift=(cz, cy, cx), axis=(0, 1, 2))
    if walls:
        for i in range(lat.q):
            cy = int(lat.c[i][1])
            if cy == 1:
                f[i, :, 1, :] = fp[lat.opp[i], :, 1, :]
            elif cy == -1:
                f[i, :, ny - 2, :] = fp[lat.opp[i], :, ny - 2, :]
        f[:, :, 0, :] = fp[:, :, 0, :]
        f[:, :, ny - 1, :] = fp[:, :, ny - 1, :]
    return f
