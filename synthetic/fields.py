"""Seeded initial velocity fields.

Shapes follow the library's layout: a velocity field is (3, nz, ny, nx) in
float64, x fastest; 2-D fields have nz = 1 and a zero z component.
"""

import numpy as np


def uniform_noise_u0(nx, ny, nz, dim, amp, seed):
    """u = U(-amp, amp) per component (z component zero in 2-D)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-amp, amp, size=(3, nz, ny, nx))
    if dim == 2:
        u[2] = 0.0
    return u


def channel_u0(nx, ny, nz, u_c, noise_frac, seed, dim=3):
    """Laminar parabola with centre-line u_c between halfway walls, plus noise.

    Rows y = 0 and y = ny-1 are the solid layers; the walls sit half a cell
    inside them.  Noise is uniform in +-noise_frac*u_c on every component of
    every fluid node.  Solid rows are zero.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 0.5 * (ny - 2)
    y = np.arange(ny) - 0.5  # distance from the lower wall plane
    prof = u_c * (1.0 - ((y - h) / h) ** 2)
    u = np.zeros((3, nz, ny, nx))
    u[0] = prof[None, :, None]
    u += rng.uniform(-noise_frac * u_c, noise_frac * u_c, size=u.shape)
    if dim == 2:
        u[2] = 0.0
    u[:, :, 0, :] = 0.0
    u[:, :, ny - 1, :] = 0.0
    return u


def initial_velocity(wl):
    """The workload's seeded initial velocity (density starts at 1 everywhere)."""
    kind = wl["init"][0]
    if kind == "noise":
        u = uniform_noise_u0(wl["nx"], wl["ny"], wl["nz"], wl["dim"], wl["init"][1], wl["seed"])
        if wl["walls"]:
            u[:, :, 0, :] = 0.0
            u[:, :, wl["ny"] - 1, :] = 0.0
        return u
    if kind == "channel":
        return channel_u0(wl["nx"], wl["ny"], wl["nz"], wl["init"][1], wl["init"][2], wl["seed"], wl["dim"])
    if kind == "rest":
        return np.zeros((3, wl["nz"], wl["ny"], wl["nx"]))
    raise ValueError(kind)
