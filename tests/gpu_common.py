"""Helpers shared by the GPU parity tests: run the CUDA library and the oracle
on the same seeded workload and compare."""

import numpy as np

import synthetic
from oracle.sim import Simulation


def nq_of(wl):
    return (len(wl["qois"]) + wl["n_mp"]) if wl["to_mode"] != "off" else 0


def lrs_inputs(wl, sigma_ref):
    c, mu, sig = synthetic.synthetic_lrs(nq_of(wl), wl["h"], wl["seed"])
    return c, mu, sig, np.asarray(sigma_ref, dtype=np.float64)


def oracle_sigma_ref(wl, steps=3):
    """RMS of the oracle's q^{n*} over a short observe-only warm-up."""
    w = dict(wl, to_mode="observe")
    sim = Simulation(w, synthetic.initial_velocity(w))
    rows = sim.run(steps)
    nq = nq_of(wl)
    return np.sqrt((rows[:, 1:1 + nq] ** 2).mean(axis=0))


def run_oracle(wl, steps, lrs=None, track=None):
    sim = Simulation(wl, synthetic.initial_velocity(wl), lrs=lrs, track_ref=track)
    rows = sim.run(steps) if steps else np.zeros((0, 2 + 3 * nq_of(wl)))
    rho, u = sim.macros()
    return sim, rows, rho, u


def run_gpu(wl, steps, lrs=None, graphs=True, track=None, chunks=None, branching=True):
    from paper_2609_32892_b300 import LbmSim, binding as B

    g = LbmSim(wl)
    g.init(synthetic.initial_velocity(wl))
    if lrs is not None:
        g.set_lrs(*lrs)
    if track is not None:
        B.lbm_set_track_reference(g.ctx, track)
    B.lbm_set_graphs(g.ctx, graphs)
    B.lbm_set_branching(g.ctx, branching)
    for n in (chunks or [steps]):
        g.step(n)
    g.sync()
    rows = g.qoi()
    rho, u = g.macros()
    return g, rows, rho, u


def rel_l2(a, b, mask=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a = a[..., mask > 0]
        b = b[..., mask > 0]
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def fluid_mask(wl):
    m = np.ones((wl["nz"], wl["ny"], wl["nx"]))
    if wl["walls"]:
        m[:, 0, :] = 0
        m[:, -1, :] = 0
    return m
