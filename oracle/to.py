"""The Tau-orthogonal SGS forcing (Sec. 4 and App. A), literally.

QoIs (Sec. 4.1):  E_R = 1/2 sum_Omega |R v|^2,  Z_R = 1/2 sum_Omega |R curl v|^2,
                  Q_j^mp = sum_Omega w_j(y) v_x  (Eq. mean-profile-qoi),
with the integral a plain sum over fluid nodes (dx = 1).
Sensitivities (App. A):  dE_R/dv = R R v;  dZ_R/dv = (d_y RRw, -d_x RRw) in 2-D
and curl(R R omega) in 3-D;  dQ_j^mp/dv = w_j(y) e_x.
Patterns (Sec. 4.2, Eq. O-from-V):  O_i = sum_j c_ij V_j with c_ii = 1 and the
orthogonality conditions sum_Omega V_i . O_j = 0 for i != j (Eq. orthogonality).
Coefficients (Eq. tau-from-dQ):  gamma_i = dQ_i / sum_Omega V_i . O_i.
SGS increment (Eq. TO-ansatz):  dv_SGS = sum_i gamma_i O_i.

Derivatives are second-order central differences (the paper states this for
WALE; the same operator is used for the curl), zero outside Omega at walls, so
that the discrete curl and its adjoint match exactly.
"""

import numpy as np

from . import filters
from .substrate import central_diff


def curl(v, dim, walls):
    """Discrete curl by central differences; 2-D returns the scalar vorticity
    d_x v_y - d_y v_x as a one-component field."""
    if dim == 2:
        return (central_diff(v[1], 0, walls) - central_diff(v[0], 1, walls))[None]
    d = lambda comp, ax: central_diff(v[comp], ax, walls)  # noqa: E731
    return np.stack([d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)])


def curl_adjoint(w, dim, walls):
    """curl^* of App. A: (d_y w, -d_x w) in 2-D; curl w in 3-D."""
    if dim == 2:
        out = np.zeros((3,) + w.shape[1:])
        out[0] = central_diff(w[0], 1, walls)
        out[1] = -central_diff(w[0], 0, walls)
        return out
    return curl(w, dim, walls)


def mp_band_weights(ny, n_bands):
    """Mean-profile band weights (Eq. 3d-mp-band-weights) on the fluid rows
    y = 1..ny-2 of a channel with halfway walls: d_w = min(y_w, 2H - y_w) with
    y_w = y - 1/2 and H = (ny - 2)/2; centres log-spaced from 0.5 (first fluid
    node) to H; sigma = the spacing of ln(centre); each band sums to 1 over
    the fluid rows.  Returns w[j, y] with zeros on the solid rows."""
    h = 0.5 * (ny - 2)
    lc = np.linspace(np.log(0.5), np.log(h), n_bands)
    sigma = (np.log(h) - np.log(0.5)) / (n_bands - 1)
    w = np.zeros((n_bands, ny))
    y = np.arange(1, ny - 1)
    yw = y - 0.5
    dw = np.minimum(yw, 2.0 * h - yw)
    for j in range(n_bands):
        b = np.exp(-0.5 * ((np.log(dw) - lc[j]) / sigma) ** 2)
        w[j, 1:ny - 1] = b / b.sum()
    return w


class TOSetup:
    """Kernels, weights and masks for one QoI set on one grid."""

    def __init__(self, dim, nx, ny, nz, walls, qois, n_mp):
        self.dim, self.walls = dim, walls
        self.qois = list(qois)
        self.n_mp = n_mp
        self.nq = len(self.qois) + n_mp
        self.mask = np.ones((nz, ny, nx))
        if walls:
            self.mask[:, 0, :] = 0.0
            self.mask[:, ny - 1, :] = 0.0
        self.kernels = {(f, s): filters.kernel(f, s, dim) for (_, f, s) in self.qois if f != "F"}
        if any(f == "F" for (_, f, _) in self.qois) and (dim != 2 or walls):
            raise ValueError("Fourier-band QoIs need a periodic 2-D grid")
        self.w_mp = mp_band_weights(ny, n_mp) if n_mp > 0 else np.zeros((0, ny))

    def filt(self, a, f, s):
        if f == "F":
            return filters.fourier_band(a, s[0], s[1])
        return filters.apply_kernel(a, self.kernels[(f, s)], self.mask, self.walls)

    def qoi_values(self, v):
        """q = Q(v) for every QoI, in order: scale QoIs then mean-profile bands."""
        vm = v * self.mask
        q = []
        for kind, f, s in self.qois:
            if kind == "E":
                rv = self.filt(vm, f, s)
                q.append(0.5 * (rv * rv).sum())
            else:
                rw = self.filt(curl(vm, self.dim, self.walls), f, s)
                q.append(0.5 * (rw * rw).sum())
        for j in range(self.n_mp):
            q.append((self.w_mp[j][None, :, None] * vm[0]).sum())
        return np.array(q)

    def sensitivities(self, v):
        """V_j = dQ_j/dv (App. A) as fields [N_Q, 3, z, y, x]."""
        vm = v * self.mask
        out = []
        for kind, f, s in self.qois:
            if kind == "E":
                out.append(self.filt(self.filt(vm, f, s), f, s))
            else:
                w = self.filt(self.filt(curl(vm, self.dim, self.walls), f, s), f, s)
                out.append(curl_adjoint(w, self.dim, self.walls) * self.mask)
        for j in range(self.n_mp):
            vj = np.zeros_like(vm)
            vj[0] = self.w_mp[j][None, :, None] * self.mask
            out.append(vj)
        return np.array(out)


def gram(vs):
    """G_ij = sum_Omega V_i . V_j (Sec. 4.2); sensitivities vanish off Omega."""
    n = len(vs)
    g = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            g[i, j] = (vs[i] * vs[j]).sum()
    return g


def gram_is_singular(g, rel=1e-14):
    """Cholesky of G with a pivot test: singular when a pivot is at or below
    rel * max diag(G) (the SGS forcing is then skipped for the step)."""
    n = len(g)
    dmax = float(np.max(np.diag(g))) if n else 0.0
    if not dmax > 0.0:
        return True
    lo = np.zeros((n, n))
    for k in range(n):
        d = g[k, k] - (lo[k, :k] ** 2).sum()
        if d <= rel * dmax:
            return True
        lo[k, k] = np.sqrt(d)
        for i in range(k + 1, n):
            lo[i, k] = (g[i, k] - (lo[i, :k] * lo[k, :k]).sum()) / lo[k, k]
    return False


def pattern_coefficients(g):
    """c_ij from the orthogonality conditions with c_ii = 1 (Sec. 4.2).

    For pattern i the unknowns are c_ik, k != i, and the conditions are
    sum_k c_ik G_jk = 0 for every j != i, i.e. sum_{k != i} G_jk c_ik = -G_ji."""
    n = len(g)
    c = np.zeros((n, n))
    for i in range(n):
        others = [k for k in range(n) if k != i]
        c[i, i] = 1.0
        if others:
            a = g[np.ix_(others, others)]
            b = -g[others, i]
            c[i, others] = np.linalg.solve(a, b)
    return c


def pattern_norms(c, g):
    """den_i = sum_Omega V_i . O_i = sum_k c_ik G_ik."""
    return (c * g).sum(axis=1)


def patterns(c, vs):
    """O_i = sum_j c_ij V_j (Eq. O-from-V)."""
    return np.einsum("ij,jazyx->iazyx", c, vs)


def sgs_increment(gamma, os):
    """dv_SGS = sum_i gamma_i O_i (Eq. TO-ansatz)."""
    return np.einsum("i,iazyx->azyx", gamma, os)
