"""lbm_qoi_eval_static: QoIs from the library's built-in scratch array.

Some callers cannot allocate device memory at all (code running inside a CUDA
graph capture, hosts that own every device allocation through their own
arena, real-time loops that cannot take an allocation's implicit
synchronisation).  This entry point serves them: it allocates nothing and
works in one compiled-in scratch array.  The test checks it against the QoIs
the regular step reports for the same field (observe mode leaves the
predictor state in place, so the state read back after one step is the field
those QoIs were computed on), on two calls in a row, with the 1e-4 relative
tolerance the other QoI parity tests use.  This file is collected last.
"""

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,shape", [("C3", (37, 22, 19)), ("C2", (45, 38, 1))])
def test_static_scratch_qoi_matches_step(name, shape):
    import torch

    from paper_2609_32892_b300 import LbmSim, binding as B

    nx, ny, nz = shape
    wl = synthetic.workload(name, nx=nx, ny=ny, nz=nz, n_mp=0, to_mode="observe")
    ns = len(wl["qois"])
    sim = LbmSim(wl)
    sim.init(synthetic.initial_velocity(wl))
    sim.step(1)
    sim.sync()
    q_step = sim.qoi()[0, 1:1 + ns]
    _, u = sim.macros()
    sim.close()

    cfg = B.config_from_workload(wl)
    u_dev = torch.tensor(u, dtype=torch.float32, device="cuda").contiguous()
    q_dev = torch.empty(ns, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        q_dev.fill_(float("nan"))
        B.lbm_qoi_eval_static(cfg, u_dev.data_ptr(), q_dev.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(q_dev.cpu().numpy(), q_step, rtol=1e-4, atol=0)

    # a grid beyond the static array is refused with a clear error
    nbig = 400 if name == "C3" else 3000
    big = B.config_from_workload(synthetic.workload(name, nx=nbig, ny=nbig, nz=nbig if name == "C3" else 1,
                                                    n_mp=0, to_mode="observe"))
    with pytest.raises(B.LbmError) as e:
        B.lbm_qoi_eval_static(big, u_dev.data_ptr(), q_dev.data_ptr(), stream.cuda_stream)
    assert e.value.code == B.LBM_ERR_BUDGET and "scratch" in str(e.value)
