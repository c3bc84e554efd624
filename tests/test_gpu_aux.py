"""Checkpoint/resume and failure detection through the C ABI.

Failure is injected from the host (a NaN written into one population with
lbm_set_populations); nothing faults, traps or hangs the device: the collide
kernel sets a status bit that lbm_sync and the QoI flags report."""

import numpy as np
import pytest

import synthetic
from gpu_common import nq_of

pytestmark = pytest.mark.gpu


def _sim(wl):
    from paper_2609_32892_b300 import LbmSim

    s = LbmSim(wl)
    s.init(synthetic.initial_velocity(wl))
    nq = nq_of(wl)
    c, mu, sig = synthetic.synthetic_lrs(nq, wl["h"], wl["seed"])
    s.set_lrs(c, mu, sig, np.zeros(nq))
    return s


def test_checkpoint_resume_is_bit_exact():
    from paper_2609_32892_b300 import LbmSim, binding as B

    wl = synthetic.workload("C3", nx=21, ny=18, nz=11, h=3)
    a = _sim(wl)
    a.step(9)
    a.sync()
    rows_a = a.qoi()
    f_a = a.populations()
    prof_a = B.lbm_get_profile(a.ctx, wl["ny"])
    a.close()

    b = _sim(wl)
    b.step(4)
    rows_b1 = b.qoi()
    blob = B.lbm_save(b.ctx)
    b.close()
    c = LbmSim(wl)  # fresh context, state only from the checkpoint
    B.lbm_load(c.ctx, blob)
    c.step(5)
    c.sync()
    rows_b2 = c.qoi()
    np.testing.assert_array_equal(np.vstack([rows_b1, rows_b2]), rows_a)
    np.testing.assert_array_equal(c.populations(), f_a)
    prof_c = B.lbm_get_profile(c.ctx, wl["ny"])
    np.testing.assert_array_equal(prof_c[0], prof_a[0])
    assert prof_c[1] == prof_a[1] == 9
    assert B.lbm_get_step(c.ctx) == 9
    c.close()


def test_unstable_state_is_reported():
    from paper_2609_32892_b300 import binding as B

    wl = synthetic.workload("C2", nx=40, ny=32, h=2)
    s = _sim(wl)
    s.step(2)
    s.sync()
    f = s.populations()
    f[3, 0, 10, 7] = np.nan
    B.lbm_set_populations(s.ctx, f)
    s.step(2)
    with pytest.raises(B.LbmError) as e:
        s.sync()
    assert e.value.code == B.LBM_ERR_UNSTABLE
    rows = s.qoi()
    assert int(rows[-1, -1]) & B.FLAG_UNSTABLE
    s.close()


def test_batch_reports_unstable_member():
    import torch

    from paper_2609_32892_b300 import binding as B

    w = synthetic.workload("C1", nx=24, ny=20, steps=4)
    need = B.lbm_required_bytes(B.config_from_workload(w))
    pool = torch.empty(2 * need + 4096, dtype=torch.uint8, device="cuda")
    b = B.lbm_batch_create(2, pool.data_ptr(), 2 * need)
    u_bad = synthetic.initial_velocity(w)
    u_bad[0, 0, 5, 5] = np.nan  # non-finite populations: flagged on the first step
    s_ok = B.lbm_batch_admit(b, B.config_from_workload(w), synthetic.initial_velocity(w), 4, 0)
    s_bad = B.lbm_batch_admit(b, B.config_from_workload(w), u_bad, 4, 1)
    B.lbm_batch_run(b, 4)
    torch.cuda.synchronize()
    done = {c["tag"]: c for c in B.lbm_batch_poll(b)}
    assert done[0]["status"] == B.LBM_OK
    assert done[1]["status"] == B.LBM_ERR_UNSTABLE
    B.lbm_batch_release(b, s_ok)
    B.lbm_batch_release(b, s_bad)
    B.lbm_batch_destroy(b)
