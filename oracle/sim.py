"""One LES time step of the fused method, composed literally (Sec. 3, Eqs.
LES-1..3; Sec. 4 predictor-corrector; Sec. 4.4 LRS).

State between steps: the post-collision populations f^p of the last step
(initially f^eq(rho0, u0)).  Step n:

  1. stream f^p (Eq. LES-3) with periodic wrap and halfway bounce-back;
  2. rho, rho u from the populations; the force density
     F = F_body + A sin(2 pi k y / ny) e_x - alpha rho u (Kolmogorov drag);
     the equilibrium velocity v = rho u / rho (EDM) or (rho u + F/2)/rho (Guo);
  3. tau_eff from the substrate (Sec. 5);
  4. relax (Eq. LES-1) and apply the body force: EDM f^{p*} = f^a +
     f^eq(v + F/rho) - f^eq(v) (Eq. LES-2 without the SGS term), or Guo;
  5. v^{p,n*} = sum_i c_i f^{p*}_i / rho: the predictor;
  6. QoIs q^{n*}, sensitivities V_j and the Gram matrix on v^{p,n*};
  7. dQ from the coefficient source (random gamma, fixed gamma, LRS, tracking);
  8. c_ij, gamma_i, dv_SGS (Sec. 4.2-4.3);
  9. f^p = f^{p*} + f^eq(rho, v^{p*} + dv_SGS) - f^eq(rho, v^{p*}), which
     telescopes with step 4 to the single-difference form of Eq. LES-2.

Each step returns the QoI block row [n, q^{n*}, dQ, gamma, flags] with flag
bit 1 = singular Gram (SGS skipped), bit 2 = unstable state.
"""

import numpy as np

from . import lbm, substrate, to
from .lattice import CS2, Lattice
from .lrs import LRSModel
from .philox import STREAM_GAMMA, STREAM_LRS, normals

FLAG_SINGULAR = 1
FLAG_UNSTABLE = 2

MODES = ("off", "observe", "gamma", "fixed", "lrs", "track")


class Simulation:
    def __init__(self, wl, u0, rho0=None, lrs=None, track_ref=None, member=0, gamma_fixed=None):
        self.wl = dict(wl)
        self.dim = wl["dim"]
        self.nx, self.ny, self.nz = wl["nx"], wl["ny"], wl["nz"]
        self.walls = bool(wl["walls"])
        self.lat = Lattice(self.dim)
        self.tau = float(wl["tau"])
        self.member = member
        self.seed = int(wl["seed"])
        self.mode = wl["to_mode"]
        assert self.mode in MODES
        self.to = None
        if self.mode != "off":
            self.to = to.TOSetup(self.dim, self.nx, self.ny, self.nz, self.walls, wl["qois"], wl["n_mp"])
        self.mask = np.ones((self.nz, self.ny, self.nx))
        if self.walls:
            self.mask[:, 0, :] = 0.0
            self.mask[:, self.ny - 1, :] = 0.0
        rho = np.ones((self.nz, self.ny, self.nx)) if rho0 is None else np.array(rho0, dtype=np.float64)
        u = np.array(u0, dtype=np.float64) * self.mask[None]
        rho = np.where(self.mask > 0, rho, 1.0)
        self.fp = lbm.equilibrium(self.lat, rho, u)
        self.lrs = None
        if self.mode == "lrs":
            c, mu, sigma, sigma_ref = lrs[:4]
            hist = lrs[4:] if len(lrs) > 4 else (None, None)
            self.lrs = LRSModel(c, mu, sigma, sigma_ref, wl["h"], *hist)
        self.track_ref = None if track_ref is None else np.asarray(track_ref, dtype=np.float64)
        # 'fixed': the caller's coefficients gamma_i, held for every step
        self.gamma_fixed = None if gamma_fixed is None else np.asarray(gamma_fixed, dtype=np.float64)
        self.n = 0
        self.profile_sum = np.zeros(self.ny)
        y = np.arange(self.ny, dtype=np.float64)
        self.kolmo = wl["kolmo_amp"] * np.sin(2.0 * np.pi * wl["kolmo_k"] * y / self.ny)

    # -- pieces -------------------------------------------------------------
    def force_density(self, rho, j):
        fx, fy, fz = self.wl["body_force"]
        f = np.zeros((3, self.nz, self.ny, self.nx))
        f[0] += fx + self.kolmo[None, :, None]
        f[1] += fy
        f[2] += fz
        f -= self.wl["kolmo_drag"] * j
        return f * self.mask[None]

    def macros(self):
        """rho and v = sum c f / rho of the current (post-collision) state."""
        rho, j = lbm.moments(self.lat, self.fp)
        return rho, j / rho[None] * self.mask[None]

    # -- the step -----------------------------------------------------------
    def step(self):
        lat, m = self.lat, self.mask
        flags = 0
        f = lbm.stream(lat, self.fp, self.walls)
        rho, j = lbm.moments(lat, f)
        force = self.force_density(rho, j)
        if self.wl["forcing"] == "guo":
            v = (j + 0.5 * force) / rho[None]
        else:
            v = j / rho[None]
        v = v * m[None]
        uu = (v * v).sum(axis=0)
        bad = (~np.isfinite(rho)) | (rho <= 0.0) | (~np.isfinite(uu)) | (uu > CS2)
        if np.any(bad & (m > 0)):
            flags |= FLAG_UNSTABLE
        feq = lbm.equilibrium(lat, rho, v)
        sub = self.wl["substrate"]
        if sub == "smag":
            tau = substrate.smagorinsky_tau_eff(lat, f, feq, rho, self.tau, self.wl["c_smag"])
        elif sub == "wale":
            tau = substrate.wale_tau_eff(v, m, self.tau, self.wl["c_wale"], self.dim, self.walls)
        else:
            tau = self.tau
        fa = lbm.relax(f, feq, tau)
        if self.wl["forcing"] == "guo":
            fps = fa + lbm.guo_source(lat, force, v, tau)
        else:
            fps = lbm.edm_forcing(lat, fa, rho, v, force / rho[None])
        rho_s, j_s = lbm.moments(lat, fps)
        vps = j_s / rho[None] * m[None]

        nq = self.to.nq if self.to is not None else 0
        qstar = np.zeros(nq)
        dq = np.zeros(nq)
        gamma = np.zeros(nq)
        fp = fps
        if self.to is not None:
            qstar = self.to.qoi_values(vps)
            vs = self.to.sensitivities(vps)
            g = to.gram(vs)
            singular = to.gram_is_singular(g)
            c = den = None
            if not singular:
                c = to.pattern_coefficients(g)
                den = to.pattern_norms(c, g)
            if self.mode == "gamma":
                z = np.array(normals(self.seed, self.member, self.n, STREAM_GAMMA, nq))
                if not singular:
                    gamma = self.wl["gamma_std"] * z
                    dq = gamma * den
            elif self.mode == "fixed":
                # gamma_i given (Eq. TO-ansatz with fixed coefficients): the
                # change it makes in Q_i is dQ_i = gamma_i sum V_i . O_i
                if not singular:
                    gamma = self.gamma_fixed.copy()
                    dq = gamma * den
            elif self.mode == "lrs" and self.n < self.wl.get("spinup", 0):
                # spin-up of an online run: nudged to the reference series
                # (Sec. 6.5 and 7.5: online runs start after tracked steps that
                # fill the history); the reference enters the history
                q = self.track_ref[min(self.n, len(self.track_ref) - 1)]
                dq = q - qstar
                self.lrs.push(q, qstar)
                if not singular:
                    gamma = dq / den
            elif self.mode == "lrs":
                z = normals(self.seed, self.member, self.n, STREAM_LRS, nq)
                q = self.lrs.predict(qstar, z)
                dq = q - qstar
                self.lrs.push(q, qstar)
                if not singular:
                    gamma = dq / den
            elif self.mode == "track":
                dq = self.track_ref[min(self.n, len(self.track_ref) - 1)] - qstar
                if not singular:
                    gamma = dq / den
            if singular:
                flags |= FLAG_SINGULAR
            elif self.mode != "observe":
                dv = to.sgs_increment(gamma, to.patterns(c, vs))
                fp = fps + lbm.equilibrium(lat, rho, vps + dv) - lbm.equilibrium(lat, rho, vps)
        if self.walls:
            fp = fp * m[None] + self.fp * (1.0 - m[None])
        self.fp = fp
        if self.to is not None:
            r, jj = lbm.moments(lat, fp)
            self.profile_sum += ((jj[0] / r) * m).sum(axis=(0, 2)) / (self.nx * self.nz)
        row = np.concatenate([[float(self.n)], qstar, dq, gamma, [float(flags)]])
        self.n += 1
        return row

    def run(self, nsteps):
        return np.array([self.step() for _ in range(nsteps)])
