"""Continuous-batching ensemble server over the C batch API (lbm_batch_*).

Requests (LES ensemble members of different grids, seeds and horizons) arrive
over time.  The server admits a request as soon as a slot and enough pool
memory are free (first come, first served), queues `chunk` steps of every
active member per round so that members admitted while others run overlap on
the device, keeps one round queued behind the running one (the device never
drains between rounds), and collects completions without blocking.  Per request it
records the queueing delay, the completion time (device clock) and the
latency per simulated time unit.

A request is a workload dict (the lbm_config fields, see binding.config_from_workload)
plus what the member needs from its caller:
  steps         horizon (lattice steps)
  u0            initial velocity, host FP64 [3][nz][ny][nx]
  steps_per_tu  lattice steps per simulated time unit (for the latency figure)
  lrs           (C, mu, Sigma, sigma_ref) of the member's LRS model (to_mode 'lrs';
                sigma_ref <= 0 entries are taken from the member's first step)
  gamma_fixed   its gamma_i (to_mode 'fixed')
  track_ref     its reference QoI series (to_mode 'track')
  arrival_s     arrival time (realtime serving)

Scheduling and marshalling only: every step runs in liblbm.so.
"""

import collections
import os
import time

import numpy as np

from . import binding as B

# Each member steps on its own stream.  With the default 8 hardware work
# queues, dozens of member streams alias onto shared queues and serialise one
# another; 32 lets them run side by side (several times the member-steps/s for
# small members).  The variable is read when the CUDA context is created, so
# it takes effect when this module is imported before the first CUDA call.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")


def set_coefficients(ctx, req):
    """The member's coefficient source from the request (lbm_set_to_coeffs)."""
    mode = req["to_mode"]
    if mode == "lrs":
        c, mu, sig, sref = req["lrs"]
        B.lbm_set_to_coeffs(ctx, "lrs", req["h"], c, mu, sig, sref)
    elif mode == "fixed":
        B.lbm_set_to_coeffs(ctx, "fixed", gamma_fixed=req["gamma_fixed"])
    elif mode == "track":
        B.lbm_set_track_reference(ctx, req["track_ref"])


class EnsembleServer:
    """persistent: lanes of persistent batched kernels per class for members
    of at most max_nodes nodes (lbm_batch_set_persistent; the library
    defaults: 1 lane, 16384 nodes); 0: per-member graphs for every member."""

    def __init__(self, pool_bytes, n_slots, device="cuda", persistent=1, max_nodes=16384):
        import torch

        self.torch = torch
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device)
        torch.cuda.synchronize(self.pool.device)
        self.batch = B.lbm_batch_create(n_slots, self.pool.data_ptr(), int(pool_bytes))
        B.lbm_batch_set_persistent(self.batch, int(persistent), max_nodes)
        torch.cuda.synchronize(self.pool.device)
        self.t_epoch = time.perf_counter()  # device time 0 of t_done_ms

    def close(self):
        if self.batch is not None:
            B.lbm_batch_destroy(self.batch)
            self.batch = None

    def admit(self, req, tag):
        cfg = B.config_from_workload(req, member=tag)
        slot = B.lbm_batch_admit(self.batch, cfg, req["u0"], req["steps"], tag)
        if slot is None:
            return None
        set_coefficients(B.lbm_batch_member(self.batch, slot), req)
        return slot

    def serve(self, requests, chunk=32, keep_qoi=False, realtime=True):
        """Run a request list (dicts with arrival_s, steps, ...) to completion.

        realtime=True honours the arrival times against the wall clock;
        False admits every request as soon as it fits (offline batch)."""
        torch = self.torch
        pending = collections.deque(sorted(range(len(requests)), key=lambda i: requests[i].get("arrival_s", 0.0)))
        active = {}
        out = {}
        t0 = time.perf_counter()
        rounds = 0
        while pending or active:
            now = time.perf_counter() - t0
            while pending:
                i = pending[0]
                r = requests[i]
                if realtime and r.get("arrival_s", 0.0) > now:
                    break
                slot = self.admit(r, i)
                if slot is None:
                    break  # head of the queue waits for memory or a slot
                active[slot] = i
                out[i] = {"arrival_s": r.get("arrival_s", 0.0) if realtime else 0.0, "admit_s": now,
                          "steps": r["steps"], "tu": r["steps"] / r["steps_per_tu"],
                          "nodes": r["nx"] * r["ny"] * r["nz"], "storage": r.get("storage", "fp32")}
                pending.popleft()
            if active:
                B.lbm_batch_run(self.batch, chunk)
                rounds += 1
                # keep one round queued behind the running one: the device is
                # never drained while the host admits and releases members
                B.lbm_batch_wait(self.batch, 1)
                for c in B.lbm_batch_poll(self.batch):
                    i = c["tag"]
                    rec = out[i]
                    rec["done_s"] = (self.t_epoch + c["t_done_ms"] * 1e-3) - t0
                    rec["status"] = c["status"]
                    if keep_qoi:
                        ctx = B.lbm_batch_member(self.batch, c["slot"])
                        rows, _ = B.lbm_qoi(ctx, 2 + 3 * (len(requests[i]["qois"]) + requests[i]["n_mp"]),
                                            capacity=max(1, requests[i]["steps"]))
                        rec["qoi"] = rows
                    B.lbm_batch_release(self.batch, c["slot"])
                    del active[c["slot"]]
            elif pending and realtime:
                time.sleep(max(0.0, min(0.01, requests[pending[0]]["arrival_s"] - now)))
        wall = time.perf_counter() - t0
        return out, wall, rounds


def summarize(out, wall):
    lat = np.array([(r["done_s"] - r["arrival_s"]) / r["tu"] for r in out.values()])
    queue = np.array([r["admit_s"] - r["arrival_s"] for r in out.values()])
    member_steps = sum(r["steps"] for r in out.values())
    node_steps = sum(r["steps"] * r["nodes"] for r in out.values())
    return {
        "requests": len(out),
        "wall_s": round(wall, 3),
        "member_steps_per_s": round(member_steps / wall, 1),
        "mlups": round(node_steps / wall / 1e6, 1),
        "latency_s_per_tu_p50": float(np.percentile(lat, 50)),
        "latency_s_per_tu_p99": float(np.percentile(lat, 99)),
        "queue_s_p50": float(np.percentile(queue, 50)),
        "queue_s_p99": float(np.percentile(queue, 99)),
        "unstable": int(sum(1 for r in out.values() if r.get("status", 0) != 0)),
    }


def serial_baseline(requests, device="cuda"):
    """One request at a time (each to completion, in arrival order): the
    throughput a one-run-at-a-time workflow gets on the same device."""
    import torch

    from .sim import LbmSim

    t0 = time.perf_counter()
    steps = 0
    nodes = 0
    unstable = 0
    for i, r in enumerate(requests):
        s = LbmSim(r, member=i, device=device)
        s.init(r["u0"])
        set_coefficients(s.ctx, r)
        s.step(r["steps"])
        try:
            s.sync()
        except B.LbmError as e:  # a member that went unstable still ran its steps
            if e.code != B.LBM_ERR_UNSTABLE:
                raise
            unstable += 1
        s.close()
        steps += r["steps"]
        nodes += r["steps"] * r["nx"] * r["ny"] * r["nz"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"requests": len(requests), "wall_s": round(wall, 3), "member_steps_per_s": round(steps / wall, 1),
            "mlups": round(nodes / wall / 1e6, 1), "unstable": unstable}
