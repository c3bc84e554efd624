"""lbm_qoi_eval_static: QoIs from the library's built-in scratch array.

Some callers cannot allocate device memory at all (code running inside a CUDA
graph capture, hosts that own every device allocation through their own
arena, real-time loops that cannot take an allocation's implicit
synchronisation).  This entry point serves them: it allocates nothing and
works in one compiled-in scratch array.  The test gives it a seeded FP32
velocity field and checks its QoIs against the FP64 oracle's QoIs of the same
field (the FP32 values widened), on two calls in a row, with the 1e-4
relative tolerance the other QoI parity tests use; it also checks them
against the existing entry point that computes the same QoIs from a context's
own scratch (lbm_eval_qoi).  Grids: ragged 3-D and 2-D ones (one-node
kernels) and a 3-D one with nx % 4 == 0 (the four-node curl and reduction
paths over the static array).  This file is collected last.
"""

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,shape", [("C3", (37, 22, 19)), ("C3", (40, 22, 19)), ("C2", (45, 38, 1))])
def test_static_scratch_qoi_matches_oracle(name, shape):
    import torch

    from oracle.to import TOSetup
    from paper_2609_32892_b300 import LbmSim, binding as B

    nx, ny, nz = shape
    wl = synthetic.workload(name, nx=nx, ny=ny, nz=nz, n_mp=0, to_mode="observe")
    ns = len(wl["qois"])
    u32 = synthetic.initial_velocity(wl).astype(np.float32)
    if wl["dim"] == 2:
        u32[2] = 0.0
    q_oracle = TOSetup(wl["dim"], nx, ny, nz, wl["walls"], wl["qois"], 0).qoi_values(u32.astype(np.float64))

    cfg = B.config_from_workload(wl)
    u_dev = torch.tensor(u32, device="cuda").contiguous()
    q_dev = torch.empty(ns, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        q_dev.fill_(float("nan"))
        B.lbm_qoi_eval_static(cfg, u_dev.data_ptr(), q_dev.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(q_dev.cpu().numpy(), q_oracle, rtol=1e-4, atol=0)

    # the existing entry point on a context's own scratch gives the same QoIs
    sim = LbmSim(wl)
    q_ctx = torch.empty(ns, dtype=torch.float64, device="cuda")
    B.lbm_eval_qoi(sim.ctx, u_dev.data_ptr(), q_ctx.data_ptr())
    torch.cuda.synchronize()
    sim.close()
    np.testing.assert_allclose(q_dev.cpu().numpy(), q_ctx.cpu().numpy(), rtol=1e-4, atol=0)

    # a grid beyond the static array is refused with a clear error
    nbig = 400 if name == "C3" else 3000
    big = B.config_from_workload(synthetic.workload(name, nx=nbig, ny=nbig, nz=nbig if name == "C3" else 1,
                                                    n_mp=0, to_mode="observe"))
    with pytest.raises(B.LbmError) as e:
        B.lbm_qoi_eval_static(big, u_dev.data_ptr(), q_dev.data_ptr(), stream.cuda_stream)
    assert e.value.code == B.LBM_ERR_BUDGET and "scratch" in str(e.value)
