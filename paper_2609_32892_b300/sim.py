"""Convenience wrapper: one simulation in a torch-allocated device buffer.

Marshalling only (allocation through torch, calls through the C ABI)."""

import numpy as np

from . import binding as B


class LbmSim:
    def __init__(self, wl, member=0, device="cuda", stream=None):
        import torch

        self.wl = dict(wl)
        self.cfg = B.config_from_workload(wl, member)
        self.nbytes = B.lbm_required_bytes(self.cfg)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.buf.device)
        self.ctx = B.lbm_create(self.cfg, self.buf.data_ptr(), self.nbytes, self.stream.cuda_stream)
        self.shape = (wl["nz"], wl["ny"], wl["nx"])
        self.q = 9 if wl["dim"] == 2 else 19
        self.row_len = B.lbm_qoi_row_len(self.cfg)

    def init(self, u0, rho0=None):
        B.lbm_init_macros(self.ctx, rho0, u0)

    def set_lrs(self, c, mu, sigma, sigma_ref, q_hist=None, qs_hist=None):
        B.lbm_set_lrs(self.ctx, c, mu, sigma, sigma_ref, q_hist, qs_hist)

    def set_to_coeffs(self, mode, h=0, c=None, mu=None, sigma=None, sigma_ref=None, gamma_fixed=None):
        B.lbm_set_to_coeffs(self.ctx, mode, h, c, mu, sigma, sigma_ref, gamma_fixed)

    def step(self, n):
        B.lbm_step(self.ctx, n)

    def sync(self):
        B.lbm_sync(self.ctx)

    def qoi(self):
        rows, lost = B.lbm_qoi(self.ctx, self.row_len)
        return rows

    def macros(self):
        return B.lbm_get_macros(self.ctx, self.shape)

    def populations(self):
        return B.lbm_get_populations(self.ctx, self.q, self.shape)

    def close(self):
        if self.ctx is not None:
            B.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nq_of(wl):
    return (len(wl["qois"]) + wl["n_mp"]) if wl["to_mode"] != "off" else 0


__all__ = ["LbmSim", "nq_of", "np"]
