"""Write the stored oracle runs that the long GPU parity tests compare against.

The FP64 oracle applies every filter as a dense kernel, so a 3-D TO-LRS run
takes seconds per step on the CPU: too slow to repeat inside a GPU test.  This
script runs it once and stores the result next to itself.  It imports only the
oracle and the seeded input generators; no value comes from the CUDA library.

Each case is a channel LES with WALE and TO-LRS forcing (the 96x40x48 workload's
physics and its 12 QoIs) on a smaller grid:

  c3_68x38x17_h20   100 steps on 68 x 38 x 17 (two full 32 x 16 filter tiles
                    in x and y plus ragged ones), h = 20: 493 rows of C, so
                    the history product spans two 256-row blocks
  c3_36x22x13_h20   1000 steps on 36 x 22 x 13, h = 20
  c3_36x22x13_h20_u0f32   the same from the initial field rounded to FP32
  c3_96x40x48_h500  6 steps of the 96x40x48 workload itself (h = 500: 12 013
                    rows of C), full-size filter tiles in every direction
  c2_256_h400       100 steps of the 256^2 Kolmogorov workload itself
                    (Smagorinsky + TO-LRS, 4 QoIs, h = 400: 3205 rows of C)

Stored per case (float64): the QoI block rows, the final density and velocity
(`Simulation.macros`), the running mean-profile sum, the reference scales.  A
case with `sample` stores the final state only on nodes x[::sx], z[::sz] (all
rows), in float32 (far below the FP32-run tolerances), to keep the file small.

Usage:  python tests/golden/make_oracle_runs.py [case ...]   (all cases by default)
"""

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_runs")

CASES = {
    "c3_68x38x17_h20": dict(name="C3", kw=dict(nx=68, ny=38, nz=17, h=20), steps=100, warm=3),
    "c3_36x22x13_h20": dict(name="C3", kw=dict(nx=36, ny=22, nz=13, h=20), steps=1000, warm=3),
    # the same run from the initial field rounded to FP32: the oracle's own
    # sensitivity to a perturbation of the size of FP32 rounding
    "c3_36x22x13_h20_u0f32": dict(name="C3", kw=dict(nx=36, ny=22, nz=13, h=20), steps=1000, warm=3, u0_f32=True),
    "c3_96x40x48_h500": dict(name="C3", kw=dict(), steps=6, warm=3, sample=(3, 2)),
    "c2_256_h400": dict(name="C2", kw=dict(), steps=100, warm=3, sample=(2, 1)),
}


def case_workload(case):
    """The workload dict of a stored case (the tests rebuild it the same way)."""
    import synthetic

    c = CASES[case]
    return synthetic.workload(c["name"], **c["kw"])


def _run(case):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    import numpy as np

    import synthetic
    from oracle.sim import Simulation

    c = CASES[case]
    wl = case_workload(case)
    nq = len(wl["qois"]) + wl["n_mp"]
    # reference scales: RMS of q^{n*} over a short observe-only warm-up
    obs = dict(wl, to_mode="observe")
    rows = Simulation(obs, synthetic.initial_velocity(obs)).run(c["warm"])
    sigma_ref = np.sqrt((rows[:, 1:1 + nq] ** 2).mean(axis=0))
    cmat, mu, sig = synthetic.synthetic_lrs(nq, wl["h"], wl["seed"])
    t0 = time.time()
    u0 = synthetic.initial_velocity(wl)
    if c.get("u0_f32"):
        u0 = u0.astype(np.float32).astype(np.float64)
    sim = Simulation(wl, u0, lrs=(cmat, mu, sig, sigma_ref))
    rows = sim.run(c["steps"])
    rho, u = sim.macros()
    if c.get("sample"):
        sx, sz = c["sample"]
        rho = rho[::sz, :, ::sx].astype(np.float32)
        u = u[:, ::sz, :, ::sx].astype(np.float32)
    np.savez_compressed(os.path.join(OUT, case + ".npz"), rows=rows, rho=rho, u=u,
                        profile_sum=sim.profile_sum, sigma_ref=sigma_ref,
                        meta=json.dumps(dict(case=case, steps=c["steps"], workload=c["name"], kw=c["kw"],
                                             sample=c.get("sample"))))
    return case, time.time() - t0, int(np.max(rows[:, -1]))


def main(names):
    os.makedirs(OUT, exist_ok=True)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(names)) as pool:
        for case, secs, flags in pool.imap_unordered(_run, names):
            print(f"{case}: {secs:.0f} s, max flags {flags}", flush=True)


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    main(sys.argv[1:] or list(CASES))
