"""The closure's workflow on the device: a tracking run supplies the training
series, the LRS model is fitted on the host, and the online run with that
model stays stable and near the reference statistics."""

import numpy as np
import pytest

import synthetic
from gpu_common import nq_of

pytestmark = pytest.mark.gpu


def test_track_fit_online():
    from paper_2609_32892_b300 import LbmSim, binding as B, train

    base = synthetic.workload("C2", nx=48, ny=40, h=3)
    nq = nq_of(base)
    # reference trajectory: an observe-only run, nudged 0.05 % upwards
    obs = LbmSim(dict(base, to_mode="observe"))
    obs.init(synthetic.initial_velocity(base))
    obs.step(300)
    qref = obs.qoi()[:, 1:1 + nq] * 1.0005
    obs.close()
    # tracking run toward it
    trk = LbmSim(dict(base, to_mode="track", track_len=len(qref)))
    trk.init(synthetic.initial_velocity(base))
    B.lbm_set_track_reference(trk.ctx, qref)
    trk.step(300)
    trk.sync()
    rows = trk.qoi()
    trk.close()
    q, qs = train.series_from_rows(rows, nq)
    np.testing.assert_allclose(q, qref, rtol=1e-12)  # tracking reaches the reference exactly in Q
    sref = qref.std(axis=0) + 1e-30
    c, mu, sig, _ = train.fit_lrs(q[50:], qs[50:], base["h"], sref, 1.0)
    sig = sig + 1e-12 * np.eye(nq) * np.trace(sig)
    # online run: spin-up on the reference, then the fitted model
    onl = LbmSim(dict(base, spinup=50, track_len=len(qref)))
    onl.init(synthetic.initial_velocity(base))
    B.lbm_set_track_reference(onl.ctx, qref)
    onl.set_lrs(c, mu, sig, sref)
    onl.step(300)
    onl.sync()
    out = onl.qoi()
    onl.close()
    assert np.all(out[:, -1] == 0)
    mean_on = out[100:, 1:1 + nq].mean(axis=0)
    mean_ref = qref[100:].mean(axis=0)
    assert np.all(np.abs(mean_on - mean_ref) <= 0.05 * np.abs(mean_ref))
