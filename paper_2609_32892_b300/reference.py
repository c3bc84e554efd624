"""HF reference QoI trajectories on the GPU (Sec. 3 coarse graining; the
reference series of Sec. 4.4 tracking and Sec. 4.5 training).

A high-fidelity (HF) run advances m HF steps per LF step; after each block of
m steps the library projects its state onto the LF lattice (lbm_project,
phi_m) and evaluates the LF QoIs on the projected velocity (lbm_eval_qoi) in
an observing LF context.  Row n holds Q(phi_m u) after (n + 1) m HF steps,
Q_ref at the end of LF step n.  Rows stay on the device until the end.

Scheduling and marshalling only: every step, projection and QoI evaluation
runs in liblbm.so.
"""

import numpy as np

import synthetic
from . import binding as B
from .sim import LbmSim


def lf_config(lf_wl, member=0):
    """The observing LF configuration of an LF workload (its QoIs, no SGS)."""
    return B.config_from_workload(dict(lf_wl, to_mode="observe", spinup=0), member=member)


class HFReference:
    """An HF run paired with an observing LF context of the projected grid."""

    def __init__(self, hf_wl, lf_wl, m, device="cuda"):
        import torch

        self.torch = torch
        self.m = int(m)
        hf_wl = dict(hf_wl, to_mode="off")
        dims = B.lbm_project_shape(B.config_from_workload(hf_wl), self.m)
        if dims != (lf_wl["nx"], lf_wl["ny"], lf_wl["nz"]):
            raise ValueError(f"phi_{m} of the HF grid is {dims}, the LF workload has "
                             f"{(lf_wl['nx'], lf_wl['ny'], lf_wl['nz'])}")
        self.hf = LbmSim(hf_wl, device=device)
        self.hf.init(synthetic.initial_velocity(hf_wl))
        self.lf_wl = dict(lf_wl, to_mode="observe", spinup=0)
        self.lf = LbmSim(self.lf_wl, device=device, stream=self.hf.stream)
        self.nq = len(lf_wl["qois"]) + lf_wl["n_mp"]
        nl = dims[0] * dims[1] * dims[2]
        dev = torch.device(device)
        self.drho = torch.empty(nl, dtype=torch.float32, device=dev)
        self.u = torch.empty(3 * nl, dtype=torch.float32, device=dev)

    def run(self, n_rows):
        """[n_rows, N_Q] reference QoIs (FP64), computed on the device."""
        torch = self.torch
        q = torch.empty((n_rows, self.nq), dtype=torch.float64, device=self.u.device)
        for n in range(n_rows):
            self.hf.step(self.m)
            B.lbm_project(self.hf.ctx, self.m, self.drho.data_ptr(), self.u.data_ptr())
            B.lbm_eval_qoi(self.lf.ctx, self.u.data_ptr(), q[n].data_ptr())
        self.hf.sync()
        return q.cpu().numpy()

    def projected(self):
        """(rho, u) of phi_m of the current HF state, on the host (FP64)."""
        B.lbm_project(self.hf.ctx, self.m, self.drho.data_ptr(), self.u.data_ptr())
        self.hf.sync()
        rho = 1.0 + self.drho.double().cpu().numpy()
        u = self.u.double().cpu().numpy().reshape(3, -1)
        return rho, u

    def close(self):
        self.lf.close()
        self.hf.close()


def hf_reference(hf_wl, lf_wl, m, n_rows, device="cuda"):
    """Reference QoI series [n_rows, N_Q] of an HF run projected by phi_m."""
    r = HFReference(hf_wl, lf_wl, m, device=device)
    try:
        return r.run(n_rows)
    finally:
        r.close()


def tracking_reference(rows):
    """The reference array lbm_set_track_reference takes ([T][N_Q] FP64)."""
    return np.ascontiguousarray(rows, dtype=np.float64)
