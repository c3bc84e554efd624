"""Projection phi_m of a high-fidelity (HF) field onto an m-times coarser
lattice (Sec. 3, coarse graining: u_bar = phi_m u, rho_bar = phi_m rho), and
the HF reference QoI series built on it (the HF run, projected every m HF
steps, QoIs evaluated on the coarse grid).

Test infrastructure: the plain, slow statement of what the GPU path computes.
Only tests, the smoke check and the benchmark's CPU leg use it.

  Doubly periodic 2-D (Sec. 3, Kolmogorov case): bicubic interpolation.
    LF node (j, i) sits at the centre of its m x m block of HF nodes, HF
    coordinates (m j + (m-1)/2, m i + (m-1)/2); the value there is cubic
    convolution interpolation (Keys 1981, a = -1/2) along x and then along y
    over the four nearest HF nodes, with periodic wrap.  For odd m the centre
    is an HF node and the projection reduces to subsampling.
  Channel with walls (Sec. 3 and Sec. 7.1): wall-anchored stride-m
    subsampling.  Halfway bounce-back puts the walls half a spacing outside
    the first and last fluid rows; with H_HF = m H_LF fluid rows the LF fluid
    row j (1-based) sits m (j - 1/2) HF spacings from the wall, i.e. on HF row
    m j - (m-1)/2 (an HF node for odd m), so HF and LF walls coincide.  Along
    the periodic x and z the LF node takes the HF block centre m i + (m-1)/2.
    Solid LF rows take the solid HF rows (velocity 0).  The grid of Sec. 7.1,
    1475 x 237 x 490 with m = 5, gives 295 x 49 x 98.

Velocities are projected without rescaling: an m-times coarser lattice with
an m-times longer time step (Sec. 3) keeps lattice velocities unchanged.
"""

import numpy as np

KEYS_A = -0.5


def keys_kernel(t, a=KEYS_A):
    """Keys' cubic convolution kernel W(t): 1 at 0, 0 at the other integers,
    support |t| < 2 (Keys, IEEE TASSP 29, 1981)."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    return np.where(
        t <= 1.0,
        (a + 2.0) * t**3 - (a + 3.0) * t**2 + 1.0,
        np.where(t < 2.0, a * t**3 - 5.0 * a * t**2 + 8.0 * a * t - 4.0 * a, 0.0),
    )


def lf_shape_2d(nx, ny, m):
    if nx % m or ny % m:
        raise ValueError(f"{nx}x{ny} is not divisible by m = {m}")
    return nx // m, ny // m


def lf_shape_3d(nx, ny, nz, m):
    """LF grid of the wall-anchored subsampling (needs odd m, m | nx, nz and
    m | ny - 2)."""
    if m % 2 == 0:
        raise ValueError("wall-anchored subsampling needs odd m (the block centre must be an HF node)")
    if nx % m or nz % m or (ny - 2) % m:
        raise ValueError(f"{nx}x{ny}x{nz} does not coarsen by m = {m}")
    return nx // m, (ny - 2) // m + 2, nz // m


def _cubic_axis(a, m, axis):
    """Interpolate the periodic array `a` along `axis` at X_i = m i + (m-1)/2."""
    n = a.shape[axis]
    nl = n // m
    out_shape = list(a.shape)
    out_shape[axis] = nl
    out = np.zeros(out_shape)
    for i in range(nl):
        x = m * i + 0.5 * (m - 1)
        base = int(np.floor(x))
        t = x - base
        acc = 0.0
        for k in (-1, 0, 1, 2):
            w = float(keys_kernel(t - k))
            acc = acc + w * np.take(a, (base + k) % n, axis=axis)
        idx = [slice(None)] * a.ndim
        idx[axis] = i
        out[tuple(idx)] = acc
    return out


def project_bicubic_2d(a, m):
    """phi_m of a periodic 2-D field [..., ny, nx] (x first, then y)."""
    a = np.asarray(a, dtype=np.float64)
    lf_shape_2d(a.shape[-1], a.shape[-2], m)
    return _cubic_axis(_cubic_axis(a, m, a.ndim - 1), m, a.ndim - 2)


def anchored_rows(ny_hf, m):
    """HF row of every LF row: solid rows to solid rows, fluid row j to
    m j - (m-1)/2."""
    _, nyl, _ = lf_shape_3d(m, ny_hf, m, m)
    rows = [0] + [m * j - (m - 1) // 2 for j in range(1, nyl - 1)] + [ny_hf - 1]
    return np.array(rows)


def project_stride_3d(a, m):
    """phi_m of a channel field [..., nz, ny, nx] by wall-anchored subsampling."""
    a = np.asarray(a, dtype=np.float64)
    nz, ny, nx = a.shape[-3:]
    nxl, nyl, nzl = lf_shape_3d(nx, ny, nz, m)
    c = (m - 1) // 2
    xs = m * np.arange(nxl) + c
    zs = m * np.arange(nzl) + c
    ys = anchored_rows(ny, m)
    return a[..., zs, :, :][..., :, ys, :][..., :, :, xs]


def project(a, m, dim):
    """phi_m for the lattice's geometry: bicubic in 2-D, anchored stride in 3-D."""
    if dim == 2:
        return project_bicubic_2d(a, m)
    return project_stride_3d(a, m)


def project_macros(rho, u, m, dim):
    """(rho_bar, u_bar) of Sec. 3's coarse graining; u has 3 components."""
    rp = project(rho, m, dim)
    up = np.array([project(u[c], m, dim) for c in range(u.shape[0])])
    return rp, up


def hf_reference(hf_sim, lf_setup, m, n_rows):
    """Reference series for tracking and training: row n holds the LF QoIs of
    phi_m u after (n + 1) m HF steps (Q_ref at the end of LF step n, Sec. 4.4).

    hf_sim: an oracle Simulation of the HF run (plain BGK); lf_setup: the
    oracle TOSetup of the LF QoIs.  Returns [n_rows, N_Q]."""
    out = np.zeros((n_rows, lf_setup.nq))
    for n in range(n_rows):
        hf_sim.run(m)
        rho, u = hf_sim.macros()
        _, up = project_macros(rho, u, m, hf_sim.dim)
        out[n] = lf_setup.qoi_values(up)
    return out
