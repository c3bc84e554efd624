"""Ensemble batches: a member's results are the same alone and in a mix,
admission is bounded by the pool budget, and the continuous-batching server
runs a request stream to completion."""

import numpy as np
import pytest

import synthetic
from gpu_common import nq_of

pytestmark = pytest.mark.gpu


def _members():
    a = synthetic.workload("C2", nx=48, ny=40, h=3, steps=9, seed=11)
    b = synthetic.workload("C3", nx=20, ny=20, nz=12, h=2, steps=6, seed=12)
    c = synthetic.workload("C1", nx=30, ny=26, steps=7, seed=13, storage="fp16")
    return [a, b, c]


def _alone(wl, member):
    from paper_2609_32892_b300 import LbmSim

    s = LbmSim(wl, member=member)
    s.init(synthetic.initial_velocity(wl))
    if wl["to_mode"] == "lrs":
        nq = nq_of(wl)
        c, mu, sig = synthetic.synthetic_lrs(nq, wl["h"], wl["seed"])
        s.set_lrs(c, mu, sig, np.zeros(nq))
    s.step(wl["steps"])
    s.sync()
    rows = s.qoi()
    f = s.populations()
    s.close()
    return rows, f


@pytest.mark.parametrize("persistent", [True, False])
def test_member_results_identical_alone_and_in_mix(persistent):
    import torch

    from paper_2609_32892_b300 import binding as B

    wls = _members()
    alone = [_alone(w, i) for i, w in enumerate(wls)]
    pool_bytes = sum(B.lbm_required_bytes(B.config_from_workload(w)) for w in wls) + (1 << 20)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(4, pool.data_ptr(), pool_bytes)
    B.lbm_batch_set_persistent(b, 1 if persistent else 0, max_nodes=1 << 40)
    slots = []
    for i, w in enumerate(wls):
        s = B.lbm_batch_admit(b, B.config_from_workload(w, member=i), synthetic.initial_velocity(w), w["steps"], i)
        assert s is not None
        if w["to_mode"] == "lrs":
            nq = nq_of(w)
            c, mu, sig = synthetic.synthetic_lrs(nq, w["h"], w["seed"])
            B.lbm_set_lrs(B.lbm_batch_member(b, s), c, mu, sig, np.zeros(nq))
        slots.append(s)
    done = {}
    for _ in range(10):
        B.lbm_batch_run(b, 2)
        torch.cuda.synchronize()
        for comp in B.lbm_batch_poll(b):
            done[comp["tag"]] = comp
    assert sorted(done) == [0, 1, 2]
    for i, (w, s) in enumerate(zip(wls, slots)):
        assert done[i]["status"] == 0 and done[i]["steps"] == w["steps"]
        ctx = B.lbm_batch_member(b, s)
        q = 9 if w["dim"] == 2 else 19
        f = B.lbm_get_populations(ctx, q, (w["nz"], w["ny"], w["nx"]))
        np.testing.assert_array_equal(f, alone[i][1])
        if nq_of(w):
            rows, _ = B.lbm_qoi(ctx, 2 + 3 * nq_of(w))
            np.testing.assert_array_equal(rows, alone[i][0])
        B.lbm_batch_release(b, s)
    assert B.lbm_batch_stats(b)[2] == 0
    B.lbm_batch_destroy(b)


def test_admission_by_budget():
    import torch

    from paper_2609_32892_b300 import binding as B

    w = synthetic.workload("C2", nx=64, ny=64, h=3, steps=4)
    need = B.lbm_required_bytes(B.config_from_workload(w))
    pool_bytes = need + need // 2
    pool = torch.empty(pool_bytes + 4096, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(8, pool.data_ptr(), pool_bytes)
    s0 = B.lbm_batch_admit(b, B.config_from_workload(w), synthetic.initial_velocity(w), 4, 0)
    assert s0 is not None
    assert B.lbm_batch_admit(b, B.config_from_workload(w), synthetic.initial_velocity(w), 4, 1) is None
    B.lbm_batch_release(b, s0)
    assert B.lbm_batch_admit(b, B.config_from_workload(w), synthetic.initial_velocity(w), 4, 2) is not None
    B.lbm_batch_destroy(b)


def test_server_runs_a_request_stream():
    from paper_2609_32892_b300 import serve

    reqs = synthetic.serving_requests(10, seed=5, rate_per_s=200.0, horizon_scale=0.01)
    srv = serve.EnsembleServer(pool_bytes=2 << 30, n_slots=6)
    out, wall, rounds = srv.serve(reqs, chunk=8, keep_qoi=True)
    srv.close()
    assert len(out) == 10
    for i, r in out.items():
        assert r["status"] == 0
        assert r["done_s"] >= r["admit_s"] - 1e-3
        assert r["qoi"].shape[0] == reqs[i]["steps"]
        assert np.all(np.isfinite(r["qoi"]))
    s = serve.summarize(out, wall)
    assert s["member_steps_per_s"] > 0 and s["latency_s_per_tu_p99"] >= s["latency_s_per_tu_p50"]


def test_serving_mix_members_stay_stable_over_hundreds_of_steps():
    """The serving mix's member kinds (2-D Smagorinsky + TO-LRS with 4 QoIs,
    3-D WALE + TO-LRS with 12 QoIs, automatic reference scales) run a few
    hundred steps in one batch without an unstable flag, with finite QoIs,
    and the 4-QoI members agree with the oracle over the run."""
    import torch

    from gpu_common import run_gpu, run_oracle
    from paper_2609_32892_b300 import serve

    reqs = synthetic.serving_requests(8, 5, 1.0, 0.04)
    for r in reqs:
        r["steps"] = 300
    srv = serve.EnsembleServer(2 << 30, 16, "cuda")
    out, _, _ = srv.serve(reqs, chunk=25, keep_qoi=True, realtime=False)
    srv.close()
    assert all(r["status"] == 0 for r in out.values()), [r["status"] for r in out.values()]
    for r in out.values():
        assert np.isfinite(r["qoi"][:, 1:-1]).all()
    # a small 4-QoI member against the oracle over 150 steps
    wl = synthetic.workload("C2", nx=40, ny=32, h=5, seed=21)
    nq = nq_of(wl)
    c, mu, sig = synthetic.synthetic_lrs(nq, wl["h"], wl["seed"])
    lrs = (c, mu, sig, np.zeros(nq))
    _, rg, _, u_g = run_gpu(wl, 150, lrs=lrs)
    _, ro, _, u_o = run_oracle(wl, 150, lrs=lrs)
    assert np.all(rg[:, -1] == ro[:, -1])
    np.testing.assert_allclose(rg[:, 1:1 + nq], ro[:, 1:1 + nq], rtol=1e-3)
    torch.cuda.synchronize()


def test_batch_wait_bounds_rounds_in_flight():
    """lbm_batch_wait(b, 0) returns once every queued call has finished, so
    members that reached their horizon are reported by the next poll; out of
    range round counts are refused."""
    import torch

    from paper_2609_32892_b300 import binding as B

    wls = [synthetic.workload("C2", nx=40, ny=32, h=3, seed=31), synthetic.workload("C3", nx=20, ny=20, nz=12, h=2, seed=32)]
    pool_bytes = sum(B.lbm_required_bytes(B.config_from_workload(w)) for w in wls) + (1 << 20)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(4, pool.data_ptr(), pool_bytes)
    for i, w in enumerate(wls):
        s = B.lbm_batch_admit(b, B.config_from_workload(w, member=i), synthetic.initial_velocity(w), 6, i)
        nq = nq_of(w)
        c, mu, sig = synthetic.synthetic_lrs(nq, w["h"], w["seed"])
        B.lbm_set_lrs(B.lbm_batch_member(b, s), c, mu, sig, np.zeros(nq))
    B.lbm_batch_wait(b, 1)  # nothing queued yet: returns at once
    for _ in range(2):
        B.lbm_batch_run(b, 3)
        B.lbm_batch_wait(b, 1)
    B.lbm_batch_wait(b, 0)
    done = B.lbm_batch_poll(b)
    assert sorted(d["tag"] for d in done) == [0, 1]
    assert all(d["status"] == 0 and d["steps"] == 6 for d in done)
    for bad in (-1, 4):
        with pytest.raises(B.LbmError):
            B.lbm_batch_wait(b, bad)
    B.lbm_batch_destroy(b)


def test_server_members_carry_their_own_coefficients():
    """A request brings its own coefficient source: an LRS member with its own
    (C, mu, Sigma, sigma_ref) and a fixed-gamma member with its own gamma_i,
    served together, each equal bit for bit to the same request run alone."""
    import torch

    from paper_2609_32892_b300 import LbmSim, serve

    a = synthetic.workload("C2", nx=40, ny=32, h=3, seed=41, steps=12)
    nq = nq_of(a)
    c, mu, sig = synthetic.synthetic_lrs(nq, a["h"], 77)  # not the seed's own model
    a.update(u0=synthetic.initial_velocity(a), lrs=(c, mu, sig, np.full(nq, 0.5)), steps_per_tu=100.0)
    b = synthetic.workload("C3", nx=20, ny=22, nz=12, seed=42, steps=10, to_mode="fixed")
    b.update(u0=synthetic.initial_velocity(b), gamma_fixed=np.linspace(-1e-3, 1e-3, nq_of(b)), steps_per_tu=100.0)
    srv = serve.EnsembleServer(2 << 30, 4, "cuda")
    out, _, _ = srv.serve([a, b], chunk=4, keep_qoi=True, realtime=False)
    srv.close()
    for i, r in enumerate((a, b)):
        s = LbmSim(r, member=i)
        s.init(r["u0"])
        serve.set_coefficients(s.ctx, r)
        s.step(r["steps"])
        s.sync()
        alone = s.qoi()
        s.close()
        assert out[i]["status"] == 0
        np.testing.assert_array_equal(out[i]["qoi"], alone)
    np.testing.assert_array_equal(out[1]["qoi"][:, 1 + 2 * nq_of(b):1 + 3 * nq_of(b)],
                                  np.tile(b["gamma_fixed"], (b["steps"], 1)))
    torch.cuda.synchronize()


def _admit_all(B, b, wls, tags):
    slots = []
    for w, t in zip(wls, tags):
        s = B.lbm_batch_admit(b, B.config_from_workload(w, member=t), synthetic.initial_velocity(w), w["steps"], t)
        assert s is not None
        if w["to_mode"] == "lrs":
            nq = nq_of(w)
            c, mu, sig = synthetic.synthetic_lrs(nq, w["h"], w["seed"])
            B.lbm_set_lrs(B.lbm_batch_member(b, s), c, mu, sig, np.zeros(nq))
        slots.append(s)
    return slots


def test_persistent_classes_with_mixed_sizes_parities_and_horizons():
    """Persistent batches over two lanes: members of one class with different
    grids (so different launch grids and dynamic shared memory in one batched
    kernel), admitted between rounds (so they enter at the other population
    parity), with horizons that end inside a round, next to members above the
    node limit and a member whose step calls cuFFT (Fourier-band QoIs): those
    step on their own graphs.  Every member ends bit for bit where it ends
    alone."""
    import torch

    from paper_2609_32892_b300 import binding as B

    first = [synthetic.workload("C2", nx=48, ny=40, h=3, steps=11, seed=51),
             synthetic.workload("C2", nx=64, ny=32, h=3, steps=7, seed=52),
             synthetic.workload("C3", nx=20, ny=20, nz=12, h=2, steps=9, seed=53),
             synthetic.workload("C3", nx=24, ny=18, nz=12, h=2, steps=5, seed=54)]
    later = [synthetic.workload("C2", nx=40, ny=48, h=3, steps=6, seed=55),
             synthetic.workload("C3", nx=28, ny=20, nz=14, h=2, steps=8, seed=56),
             synthetic.workload("C2F", h=3, steps=5, seed=57)]
    wls = first + later
    alone = [_alone(w, i) for i, w in enumerate(wls)]
    pool_bytes = sum(B.lbm_required_bytes(B.config_from_workload(w)) for w in wls) + (1 << 20)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(8, pool.data_ptr(), pool_bytes)
    B.lbm_batch_set_persistent(b, 2, max_nodes=5000)  # 24x18x12 and 28x20x14 above it
    slots = _admit_all(B, b, first, range(len(first)))
    B.lbm_batch_run(b, 3)  # odd: the later members enter at the other parity
    slots += _admit_all(B, b, later, range(len(first), len(wls)))
    done = {}
    for _ in range(6):
        B.lbm_batch_run(b, 4)
        B.lbm_batch_wait(b, 1)
        for comp in B.lbm_batch_poll(b):
            done[comp["tag"]] = comp
    B.lbm_batch_wait(b, 0)
    for comp in B.lbm_batch_poll(b):
        done[comp["tag"]] = comp
    torch.cuda.synchronize()
    assert sorted(done) == list(range(len(wls)))
    for i, (w, s) in enumerate(zip(wls, slots)):
        assert done[i]["status"] == 0 and done[i]["steps"] == w["steps"], (i, done[i])
        ctx = B.lbm_batch_member(b, s)
        q = 9 if w["dim"] == 2 else 19
        f = B.lbm_get_populations(ctx, q, (w["nz"], w["ny"], w["nx"]))
        np.testing.assert_array_equal(f, alone[i][1], err_msg=f"member {i}")
        rows, _ = B.lbm_qoi(ctx, 2 + 3 * nq_of(w))
        np.testing.assert_array_equal(rows, alone[i][0], err_msg=f"member {i}")
        B.lbm_batch_release(b, s)
    B.lbm_batch_destroy(b)


def test_persistent_mode_is_set_before_the_first_round():
    import torch

    from paper_2609_32892_b300 import binding as B

    w = synthetic.workload("C2", nx=32, ny=32, h=3, steps=4, seed=61)
    need = B.lbm_required_bytes(B.config_from_workload(w)) + (1 << 20)
    pool = torch.empty(need, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(2, pool.data_ptr(), need)
    _admit_all(B, b, [w], [0])
    B.lbm_batch_run(b, 2)
    with pytest.raises(B.LbmError) as e:
        B.lbm_batch_set_persistent(b, 0)
    assert e.value.code == B.LBM_ERR_STATE
    B.lbm_batch_wait(b, 0)
    B.lbm_batch_destroy(b)


def test_persistent_blocks_running_many_items_match_plain_launches():
    """Serving-mix sizes in persistent kernels: 4 x 256^2 Kolmogorov and 6 x
    96x40x48 channel members give each batched launch several times more
    work items than its persistent grid has blocks, so blocks run many items
    in a row (shared memory, mbarrier phases and bulk-copy rings reused from
    item to item).  Every member ends bit for bit where it ends alone."""
    import torch

    from paper_2609_32892_b300 import binding as B

    wls = [synthetic.workload("C2", h=5, steps=6, seed=71 + i) for i in range(4)]
    wls += [synthetic.workload("C3", h=5, steps=6, seed=81 + i) for i in range(6)]
    alone = [_alone(w, i) for i, w in enumerate(wls)]
    pool_bytes = sum(B.lbm_required_bytes(B.config_from_workload(w)) for w in wls) + (1 << 22)
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(len(wls), pool.data_ptr(), pool_bytes)
    B.lbm_batch_set_persistent(b, 1, max_nodes=1 << 40)
    slots = _admit_all(B, b, wls, range(len(wls)))
    B.lbm_batch_run(b, 6)
    B.lbm_batch_wait(b, 0)
    done = {c["tag"]: c for c in B.lbm_batch_poll(b)}
    torch.cuda.synchronize()
    for i, (w, s) in enumerate(zip(wls, slots)):
        assert done[i]["status"] == 0 and done[i]["steps"] == 6
        ctx = B.lbm_batch_member(b, s)
        q = 9 if w["dim"] == 2 else 19
        f = B.lbm_get_populations(ctx, q, (w["nz"], w["ny"], w["nx"]))
        np.testing.assert_array_equal(f, alone[i][1], err_msg=f"member {i}")
        rows, _ = B.lbm_qoi(ctx, 2 + 3 * nq_of(w))
        np.testing.assert_array_equal(rows, alone[i][0], err_msg=f"member {i}")
    B.lbm_batch_destroy(b)
