"""Projection phi_m, QoIs of a given field and the HF reference series on the
GPU against the oracle (Sec. 3 coarse graining, Sec. 4.4 tracking).

Every input is generated on the host (synthetic populations, velocities,
workloads); the oracle never sees a value the CUDA path produced.
"""

import numpy as np
import pytest

import synthetic
from gpu_common import fluid_mask, nq_of, rel_l2, run_gpu, run_oracle
from oracle import lbm as olbm
from oracle import projection as P
from oracle.lattice import Lattice
from oracle.sim import Simulation
from oracle.to import TOSetup

pytestmark = pytest.mark.gpu


def _host_state(wl, seed):
    """Equilibrium of a smooth random (rho, u) plus a small non-equilibrium part."""
    lat = Lattice(wl["dim"])
    rng = np.random.default_rng(seed)
    shape = (wl["nz"], wl["ny"], wl["nx"])
    u = 0.05 * rng.standard_normal((3,) + shape)
    if wl["dim"] == 2:
        u[2] = 0.0
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    if wl["walls"]:
        u[:, :, 0, :] = 0.0
        u[:, :, -1, :] = 0.0
        rho[:, 0, :] = 1.0
        rho[:, -1, :] = 1.0
    f = olbm.equilibrium(lat, rho, u)
    f += 1e-4 * rng.standard_normal(f.shape) * lat.w.reshape((-1,) + (1,) * 3)
    return lat, f


def _gpu_project(wl, f, m):
    import torch
    from paper_2609_32892_b300 import LbmSim, binding as B

    g = LbmSim(dict(wl, to_mode="off"))
    B.lbm_set_populations(g.ctx, f)
    dims = B.lbm_project_shape(g.cfg, m)
    nl = dims[0] * dims[1] * dims[2]
    drho = torch.full((nl,), float("nan"), dtype=torch.float32, device="cuda")
    u = torch.full((3 * nl,), float("nan"), dtype=torch.float32, device="cuda")
    B.lbm_project(g.ctx, m, drho.data_ptr(), u.data_ptr())
    g.sync()
    shape = (dims[2], dims[1], dims[0])
    out = (1.0 + drho.double().cpu().numpy().reshape(shape), u.double().cpu().numpy().reshape((3,) + shape))
    g.close()
    return out


@pytest.mark.parametrize("name,kw,m", [
    ("C2", dict(nx=48, ny=40), 4),     # even m: 4 x 4 bicubic taps, periodic wrap
    ("C2", dict(nx=45, ny=30), 3),     # odd m: block-centre subsampling
    ("C2", dict(nx=20, ny=16), 1),     # identity
    ("C3", dict(nx=27, ny=23, nz=15), 3),
    ("C3", dict(nx=25, ny=27, nz=15), 5),
])
def test_projection_matches_oracle(name, kw, m):
    wl = synthetic.workload(name, **kw)
    lat, f = _host_state(wl, 11 + m)
    rho, j = olbm.moments(lat, f)
    u = j / rho[None]
    if wl["walls"]:
        u[:, :, 0, :] = 0.0
        u[:, :, -1, :] = 0.0
        rho[:, 0, :] = 1.0
        rho[:, -1, :] = 1.0
    ro, uo = P.project_macros(rho, u, m, wl["dim"])
    rg, ug = _gpu_project(wl, f, m)
    assert rg.shape == ro.shape and ug.shape == uo.shape
    # FP32 storage of the populations and FP32 sums: absolute errors ~1e-7
    np.testing.assert_allclose(rg, ro, rtol=0, atol=2e-6)
    np.testing.assert_allclose(ug, uo, rtol=0, atol=2e-6)


def test_projection_rejects_bad_factor():
    from paper_2609_32892_b300 import binding as B

    for wl, m in [(synthetic.workload("C3", nx=24, ny=23, nz=12), 2),   # even m in 3-D
                  (synthetic.workload("C3", nx=25, ny=24, nz=10), 5),   # ny - 2 not divisible
                  (synthetic.workload("C2", nx=30, ny=32), 4)]:         # nx not divisible
        with pytest.raises(B.LbmError):
            B.lbm_project_shape(B.config_from_workload(wl), m)


@pytest.mark.parametrize("name,kw", [("C2", dict(nx=44, ny=36)), ("C3", dict(nx=33, ny=22, nz=13)),
                                     ("C3", dict(nx=36, ny=22, nz=60)),
                                     ("C3", dict(nx=36, ny=20, nz=14, walls=False, n_mp=0)), ("C2F", dict())])
def test_eval_qoi_matches_oracle(name, kw):
    """Q(u) of a host velocity field: scale QoIs (G, L, Fourier bands) and
    mean-profile bands.  nx = 33 takes the register-prefetch 3-D Laplacian
    kernels, nx = 36 the factorised / asynchronously staged ones (nx % 4 == 0),
    with nz = 60 split into three z segments per block column; the periodic
    3-D case wraps the staged y halo instead of zero-filling it."""
    import torch
    from paper_2609_32892_b300 import LbmSim, binding as B

    wl = synthetic.workload(name, to_mode="observe", **kw)
    u = synthetic.initial_velocity(dict(wl, init=("noise", 0.05)))
    if wl["walls"]:
        u = u + synthetic.initial_velocity(dict(wl, init=("channel", 0.1, 0.0)))
    setup = TOSetup(wl["dim"], wl["nx"], wl["ny"], wl["nz"], wl["walls"], wl["qois"], wl["n_mp"])
    qo = setup.qoi_values(u)
    g = LbmSim(wl)
    ud = torch.tensor(np.ascontiguousarray(u, dtype=np.float32).reshape(-1), device="cuda")
    q = torch.full((setup.nq,), float("nan"), dtype=torch.float64, device="cuda")
    B.lbm_eval_qoi(g.ctx, ud.data_ptr(), q.data_ptr())
    g.sync()
    np.testing.assert_allclose(q.cpu().numpy(), qo, rtol=2e-5, atol=0)
    g.close()


@pytest.mark.parametrize("hf,lf,m,rows", [
    (("C2", dict(nx=192, ny=192, to_mode="off", substrate="none")), ("C2", dict(nx=48, ny=48)), 4, 3),
    (("C4", dict(nx=45, ny=44, nz=27)), ("C3", dict(nx=15, ny=16, nz=9)), 3, 3),
])
def test_hf_reference_series_matches_oracle(hf, lf, m, rows):
    """The whole reference pipeline: HF run, phi_m every m steps, LF QoIs."""
    from paper_2609_32892_b300.reference import hf_reference

    hf_wl = synthetic.workload(hf[0], **hf[1])
    lf_wl = synthetic.workload(lf[0], **lf[1])
    ref_g = hf_reference(hf_wl, lf_wl, m, rows)
    sim = Simulation(dict(hf_wl, to_mode="off"), synthetic.initial_velocity(hf_wl))
    setup = TOSetup(lf_wl["dim"], lf_wl["nx"], lf_wl["ny"], lf_wl["nz"], lf_wl["walls"], lf_wl["qois"],
                    lf_wl["n_mp"])
    ref_o = P.hf_reference(sim, setup, m, rows)
    assert ref_g.shape == ref_o.shape == (rows, nq_of(lf_wl))
    np.testing.assert_allclose(ref_g, ref_o, rtol=1e-4, atol=0)


def test_tracking_a_projected_reference():
    """An LF run tracking the reference the GPU generated agrees with the
    oracle's LF run tracking the oracle's reference."""
    from paper_2609_32892_b300.reference import hf_reference

    hf_wl = synthetic.workload("C2", nx=192, ny=192, to_mode="off", substrate="none")
    lf_wl = synthetic.workload("C2", nx=48, ny=48, to_mode="track", track_len=6)
    m, steps = 4, 6
    ref_g = hf_reference(hf_wl, lf_wl, m, steps)
    sim = Simulation(dict(hf_wl, to_mode="off"), synthetic.initial_velocity(hf_wl))
    setup = TOSetup(2, 48, 48, 1, False, lf_wl["qois"], 0)
    ref_o = P.hf_reference(sim, setup, m, steps)
    _, rg, rho_g, u_g = run_gpu(lf_wl, steps, track=ref_g)
    _, ro, rho_o, u_o = run_oracle(lf_wl, steps, track=ref_o)
    assert rel_l2(u_g, u_o, fluid_mask(lf_wl)) < 1e-4
    nq = nq_of(lf_wl)
    np.testing.assert_allclose(rg[:, 1:1 + nq], ro[:, 1:1 + nq], rtol=1e-4)
    assert np.all(rg[:, -1] == 0)
