"""Pins of the full oracle step against invariants and closed forms."""

import math

import numpy as np
import pytest

import synthetic
from oracle import lbm, substrate
from oracle.lattice import CS2, Lattice
from oracle.sim import FLAG_SINGULAR, Simulation


def _lrs_inputs(wl, sigma_ref=None):
    nq = len(wl["qois"]) + wl["n_mp"]
    c, mu, sig = synthetic.synthetic_lrs(nq, wl["h"], wl["seed"])
    if sigma_ref is None:
        sigma_ref = np.ones(nq)
    return (c, mu, sig, sigma_ref)


def _sigma_ref(wl, steps=3):
    """RMS of q^{n*} over a short observe-only warm-up (the recipe for the
    synthetic LRS reference scales)."""
    w = dict(wl, to_mode="observe")
    sim = Simulation(w, synthetic.initial_velocity(w))
    rows = sim.run(steps)
    nq = len(wl["qois"]) + wl["n_mp"]
    return np.sqrt((rows[:, 1:1 + nq] ** 2).mean(axis=0))


def _total_mass(sim):
    return (sim.fp * sim.mask[None]).sum()


@pytest.mark.parametrize("case", ["c1", "c2", "c3"])
def test_mass_conserved(case):
    """BGK, EDM/Guo forcing, the SGS increment (sum delta f = 0, Sec. 3) and
    bounce-back all conserve mass: the total stays constant to 1e-12."""
    if case == "c1":
        wl = synthetic.workload("C1", nx=20, ny=16)
        lrs = None
        n = 200
    elif case == "c2":
        wl = synthetic.workload("C2", nx=24, ny=20, h=3, tau=0.51)
        lrs = _lrs_inputs(wl, _sigma_ref(wl))
        n = 60
    else:
        wl = synthetic.workload("C3", nx=8, ny=16, nz=6, h=2)
        lrs = _lrs_inputs(wl, _sigma_ref(wl, 2))
        n = 12
    sim = Simulation(wl, synthetic.initial_velocity(wl), lrs=lrs)
    m0 = _total_mass(sim)
    rows = sim.run(n)
    assert abs(_total_mass(sim) - m0) <= 1e-12 * m0
    assert np.all(rows[:, -1] == 0)  # neither singular nor unstable


def test_momentum_change_equals_force():
    """Periodic, EDM, no SGS: the total momentum grows by sum F per step."""
    wl = synthetic.workload("C1", nx=12, ny=10, forcing="edm", to_mode="off", body_force=(1e-5, -2e-6, 0.0))
    sim = Simulation(wl, synthetic.initial_velocity(wl))
    lat = sim.lat
    _, j0 = lbm.moments(lat, sim.fp)
    y = np.arange(10)
    ftot = np.array([1e-5 * 120 + (1e-5 * np.sin(2 * np.pi * 4 * y / 10)).sum() * 12, -2e-6 * 120, 0.0])
    for _ in range(5):
        sim.step()
        _, j1 = lbm.moments(lat, sim.fp)
        np.testing.assert_allclose(j1.sum(axis=(1, 2, 3)) - j0.sum(axis=(1, 2, 3)), ftot, atol=1e-16)
        j0 = j1


def test_sgs_increment_moments():
    """delta f = f^eq(rho, v + dv) - f^eq(rho, v): sum delta f = 0 and
    sum c delta f = rho dv (Sec. 3)."""
    rng = np.random.default_rng(0)
    for dim in (2, 3):
        lat = Lattice(dim)
        rho = 1 + 0.01 * rng.normal(size=(2, 3, 4))
        v = 0.05 * rng.normal(size=(3, 2, 3, 4))
        dv = 1e-3 * rng.normal(size=(3, 2, 3, 4))
        if dim == 2:
            v[2] = dv[2] = 0
        df = lbm.equilibrium(lat, rho, v + dv) - lbm.equilibrium(lat, rho, v)
        r, j = lbm.moments(lat, df)
        np.testing.assert_allclose(r, 0, atol=1e-15)
        np.testing.assert_allclose(j, rho * dv, atol=1e-15)


def test_two_stage_forcing_equals_single_difference():
    """f^a + f^eq(v + du_F + dv_SGS) - f^eq(v) (Eq. LES-2) equals the two-stage
    form f^{p*} + f^eq(v* + dv) - f^eq(v*) with f^{p*} = f^a + f^eq(v + du_F) - f^eq(v)."""
    rng = np.random.default_rng(1)
    lat = Lattice(3)
    rho = 1 + 0.01 * rng.normal(size=(2, 3, 4))
    v = 0.05 * rng.normal(size=(3, 2, 3, 4))
    duf = 1e-4 * rng.normal(size=v.shape)
    dvs = 1e-3 * rng.normal(size=v.shape)
    fa = lbm.equilibrium(lat, rho, v) + 1e-4 * rng.normal(size=(19, 2, 3, 4))
    one = fa + lbm.equilibrium(lat, rho, v + duf + dvs) - lbm.equilibrium(lat, rho, v)
    fps = lbm.edm_forcing(lat, fa, rho, v, duf)
    two = fps + lbm.equilibrium(lat, rho, v + duf + dvs) - lbm.equilibrium(lat, rho, v + duf)
    np.testing.assert_allclose(one, two, atol=1e-15)


def test_rest_state_is_a_fixed_point():
    """f = w_i with no force stays put (to rounding: the paper's relaxation
    (1 - 1/tau) f + f^eq/tau is not exact in floating point); at v = 0 every
    sensitivity vanishes, so the Gram matrix is singular and the SGS step is
    skipped."""
    wl = synthetic.workload("C3", nx=6, ny=16, nz=5, h=2, body_force=(0, 0, 0), init=("rest",))
    sim = Simulation(wl, np.zeros((3, 5, 16, 6)), lrs=_lrs_inputs(wl))
    f0 = sim.fp.copy()
    rows = sim.run(3)
    assert np.max(np.abs(sim.fp - f0)) < 1e-15
    assert np.all(rows[:, -1] == FLAG_SINGULAR)


def _physical_velocity(sim, force):
    """(sum c f + F/2)/rho from the post-collision state: v^p - F/(2 rho)."""
    rho, v = sim.macros()
    return v - 0.5 * force / rho[None] * sim.mask[None]


def _poiseuille_error(ny, tau, steps):
    fx = 1e-6
    wl = synthetic.workload("C1", nx=3, ny=ny, walls=True, tau=tau, forcing="guo", kolmo_amp=0.0,
                            to_mode="off", body_force=(fx, 0.0, 0.0), init=("rest",))
    sim = Simulation(wl, np.zeros((3, 1, ny, 3)))
    sim.run(steps)
    force = np.zeros((3, 1, ny, 3))
    force[0] = fx * sim.mask
    u = _physical_velocity(sim, force)[0, 0, 1:ny - 1, 0]
    nu = CS2 * (tau - 0.5)
    yw = np.arange(1, ny - 1) - 0.5
    exact = fx / (2 * nu) * yw * ((ny - 2) - yw)
    return np.max(np.abs(u - exact)) / np.max(exact)


def test_poiseuille_second_order_and_exact_at_magic_tau():
    """Body-force driven channel with halfway walls: parabola F y(2H-y)/(2 nu).
    BGK's wall-slip error shrinks ~4x per grid doubling; at
    tau = 1/2 + sqrt(3)/4 ((tau-1/2)^2 = 3/16) the profile is exact."""
    tau = 0.8
    e1 = _poiseuille_error(10, tau, 3000)
    e2 = _poiseuille_error(18, tau, 9000)
    assert e1 > 1e-4 and 3.0 < e1 / e2 < 5.5
    assert _poiseuille_error(10, 0.5 + math.sqrt(3) / 4, 2500) < 1e-9


def _kolmogorov_error(ny, steps_tu):
    tau, amp = 0.8, 1e-6
    nu = CS2 * (tau - 0.5)
    k = 2 * np.pi / ny
    steps = int(round(steps_tu / (nu * k * k)))
    wl = synthetic.workload("C1", nx=2, ny=ny, tau=tau, kolmo_amp=amp, kolmo_k=1, to_mode="off", init=("rest",))
    sim = Simulation(wl, np.zeros((3, 1, ny, 2)))
    sim.run(steps)
    y = np.arange(ny)
    force = np.zeros((3, 1, ny, 2))
    force[0] = (amp * np.sin(k * y))[None, :, None]
    u = _physical_velocity(sim, force)[0, 0, :, 0]
    exact = amp / (nu * k * k) * (1 - np.exp(-nu * k * k * steps)) * np.sin(k * y)
    return np.max(np.abs(u - exact)) / np.max(np.abs(exact))


def test_laminar_kolmogorov_closed_form():
    """Start from rest under A sin(k y) e_x: u_x = A/(nu k^2)(1 - exp(-nu k^2 t)) sin(k y);
    the lattice error is O(k^2): about 4x smaller per grid doubling."""
    e1 = _kolmogorov_error(16, 1.0)
    e2 = _kolmogorov_error(32, 1.0)
    assert e1 < 0.05 and 3.0 < e1 / e2 < 5.0


def _taylor_green_rate_error(n):
    tau, u0 = 0.6, 1e-4
    nu = CS2 * (tau - 0.5)
    k = 2 * np.pi / n
    x = np.arange(n)
    xx, yy = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((3, 1, n, n))
    u[0, 0] = -u0 * np.cos(k * xx) * np.sin(k * yy)
    u[1, 0] = u0 * np.sin(k * xx) * np.cos(k * yy)
    wl = synthetic.workload("C1", nx=n, ny=n, tau=tau, kolmo_amp=0.0, forcing="edm", to_mode="off")
    sim = Simulation(wl, u)
    t1, t2 = int(0.2 / (nu * k * k)), int(0.6 / (nu * k * k))
    sim.run(t1)
    e1 = (sim.macros()[1] ** 2).sum()
    sim.run(t2 - t1)
    e2 = (sim.macros()[1] ** 2).sum()
    rate = -math.log(e2 / e1) / (t2 - t1)
    return abs(rate - 4 * nu * k * k) / (4 * nu * k * k)


def test_taylor_green_energy_decay():
    """Energy of the 2-D Taylor-Green vortex decays as exp(-4 nu k^2 t)."""
    e1 = _taylor_green_rate_error(12)
    e2 = _taylor_green_rate_error(24)
    assert e1 < 0.05 and e2 < e1 / 2.5


def test_smagorinsky_solves_its_implicit_definition():
    """tau_eff = tau + nu_t/c_s^2 with nu_t = C^2 sqrt(2 S:S) and
    S = -Pi^neq / (2 rho c_s^2 tau_eff) (Sec. 5.1): the closed form satisfies it;
    nu_t = 0 at equilibrium."""
    rng = np.random.default_rng(2)
    for dim in (2, 3):
        lat = Lattice(dim)
        rho = 1 + 0.01 * rng.normal(size=(2, 3, 4))
        u = 0.05 * rng.normal(size=(3, 2, 3, 4))
        if dim == 2:
            u[2] = 0
        feq = lbm.equilibrium(lat, rho, u)
        f = feq + 1e-3 * rng.normal(size=feq.shape)
        cs, tau = 0.13, 0.51
        te = substrate.smagorinsky_tau_eff(lat, f, feq, rho, tau, cs)
        pi = np.einsum("qa,qb,qzyx->abzyx", lat.cf, lat.cf, f - feq)
        s = -pi / (2 * rho * CS2 * te)
        nut = cs * cs * np.sqrt(2 * (s * s).sum(axis=(0, 1)))
        np.testing.assert_allclose(te, tau + nut / CS2, rtol=1e-13)
        np.testing.assert_allclose(substrate.smagorinsky_tau_eff(lat, feq, feq, rho, tau, cs), tau, rtol=0, atol=0)


def test_wale_closed_form_and_pure_shear():
    """v = (A sin ky, B sin kx, 0): g_xy = A sin k cos ky, g_yx = B sin k cos kx,
    hence (by hand from Sec. 5.2) S^d:S^d = 2/3 (g_xy g_yx)^2, S:S = (g_xy + g_yx)^2/2.
    Pure shear (B = 0) gives nu_t = 0."""
    n = 16
    k = 2 * np.pi / n
    x = np.arange(n)
    xx, yy = np.meshgrid(x, x, indexing="xy")
    a_amp, b_amp, cw, tau = 0.02, 0.013, 0.5, 0.55
    v = np.zeros((3, 1, n, n))
    v[0, 0] = a_amp * np.sin(k * yy)
    v[1, 0] = b_amp * np.sin(k * xx)
    mask = np.ones((1, n, n))
    te = substrate.wale_tau_eff(v, mask, tau, cw, 2, False)[0]
    a = a_amp * np.sin(k) * np.cos(k * yy)
    b = b_amp * np.sin(k) * np.cos(k * xx)
    sdsd = (2.0 / 3.0) * (a * b) ** 2
    ss = (a + b) ** 2 / 2
    den = ss ** 2.5 + sdsd ** 1.25
    nut = np.where(den < 1e-30, 0.0, cw * cw * sdsd ** 1.5 / np.where(den < 1e-30, 1, den))
    np.testing.assert_allclose(te, tau + 3 * nut, rtol=1e-12, atol=1e-15)
    v[1] = 0
    np.testing.assert_allclose(substrate.wale_tau_eff(v, mask, tau, cw, 2, False), tau, atol=1e-18)


def test_unit_conversions_match_the_paper(root):
    """Sec. 6.2: 1.4e3 LF steps per TU at N = 128, 2.3e4 at N = 2048;
    Sec. 7.1: 4289 LF steps per TU (N_y = 49) and 21 445 HF steps (N_y = 237).
    The printed values live in tests/golden/paper_values.json."""
    import json
    import os

    g = json.load(open(os.path.join(root, "tests", "golden", "paper_values.json")))
    e = g["kolmogorov_lf_steps_per_tu"]
    assert round(synthetic.kolmogorov_lattice(e["n"])["steps_per_tu"], e["round_to"]) == e["value"]
    e = g["kolmogorov_dns_steps_per_tu"]
    assert round(synthetic.kolmogorov_lattice(e["n"])["steps_per_tu"], e["round_to"]) == e["value"]
    e = g["channel_lf_steps_per_tu"]
    assert round(synthetic.channel_lattice(e["ny"])["steps_per_tu"]) == e["value"]
    e = g["channel_hf_steps_per_tu"]
    assert abs(synthetic.channel_lattice(e["ny"])["steps_per_tu"] / e["value"] - 1) < e["rel_tol"]
    c3 = synthetic.channel_lattice(40)
    assert abs(c3["tau"] - 0.50173) < 1e-5


def test_printed_filter_constants(root):
    """The filter constants printed in Sec. 4.1 (golden file) hold for the oracle kernels."""
    import json
    import os

    from oracle import filters

    g = json.load(open(os.path.join(root, "tests", "golden", "paper_values.json")))
    assert list(filters.ELL) == g["biharmonic_stencil"]["value"]
    for dim, key in [(2, "2d"), (3, "3d")]:
        assert filters.gaussian_kernel(3, dim).shape[0] == 2 * 3 * g["gaussian_alpha"][key] + 1
        for s in (1, 3):
            assert abs(np.abs(filters.laplacian_kernel(s, dim)).sum() - g["laplacian_abs_sum"]["value"]) < 1e-14


def test_lrs_spin_up_follows_the_reference():
    """During the spin-up of an online run, dQ = Q_ref - q* and the reference
    (not an LRS prediction) enters the corrected-QoI history; afterwards the
    LRS model takes over.  The reference is the observed run's own predictor
    QoIs raised by 1e-4, a nudge small enough that every step stays stable."""
    wl = synthetic.workload("C2", nx=20, ny=18, h=3, spinup=2, track_len=2)
    nq = len(wl["qois"])
    u0 = synthetic.initial_velocity(wl)
    obs = Simulation(dict(wl, to_mode="observe", spinup=0), u0).run(2)
    ref = obs[:, 1:1 + nq] * (1.0 + 1e-4)
    sim = Simulation(wl, u0, lrs=_lrs_inputs(wl, _sigma_ref(wl)), track_ref=ref)
    rows = sim.run(3)
    assert np.all(rows[:, -1] == 0)  # neither singular nor unstable
    assert np.all(np.isfinite(rows)) and np.all(np.isfinite(sim.fp))
    q, dq = rows[:, 1:1 + nq], rows[:, 1 + nq:1 + 2 * nq]
    # step 0 starts from the observed run's state: the same predictor QoIs
    np.testing.assert_array_equal(q[0], obs[0, 1:1 + nq])
    # spin-up steps: dQ = Q_ref - q*, a nudge of about 1e-4 q*
    np.testing.assert_allclose(dq[:2], ref - q[:2], rtol=1e-15)
    assert np.all(np.abs(dq[0]) > 0.5e-4 * np.abs(q[0]))
    # histories, most recent first: the LRS prediction of step 2, then the references
    np.testing.assert_array_equal(sim.lrs.q_hist[1], ref[1])
    np.testing.assert_array_equal(sim.lrs.q_hist[2], ref[0])
    np.testing.assert_allclose(sim.lrs.q_hist[0] - q[2], dq[2], rtol=0, atol=1e-15 * np.abs(q[2]).max())
    np.testing.assert_array_equal(sim.lrs.qs_hist[0], q[2])
    np.testing.assert_array_equal(sim.lrs.qs_hist[1], q[1])


def test_fixed_gamma_moves_each_qoi_by_gamma_times_its_pattern_norm():
    """Fixed coefficients (Eq. TO-ansatz with caller-given gamma_i): the step
    adds f^eq(rho, v* + dv) - f^eq(rho, v*), which shifts the velocity by
    exactly dv, so dv is read off the two states (the fixed-gamma step and
    an observed step from the same start).  Then <V_j, dv> = gamma_j <V_j, O_j>
    (orthogonal patterns) = dQ_j of the QoI row, for every j."""
    wl = synthetic.workload("C2", nx=22, ny=20, to_mode="fixed")
    nq = len(wl["qois"])
    u0 = synthetic.initial_velocity(wl)
    gam = np.array([2e-3, -1e-3, 5e-4, 1.5e-3])[:nq]
    fixed = Simulation(wl, u0, gamma_fixed=gam)
    row = fixed.run(1)[0]
    obs = Simulation(dict(wl, to_mode="observe"), u0)
    obs.run(1)
    assert row[-1] == 0
    np.testing.assert_array_equal(row[1 + 2 * nq:1 + 3 * nq], gam)
    _, v_fix = fixed.macros()
    _, v_obs = obs.macros()  # v^{p*} of the same step
    dv = v_fix - v_obs
    vs = fixed.to.sensitivities(v_obs)
    proj = np.array([(vs[j] * dv).sum() for j in range(nq)])
    dq = row[1 + nq:1 + 2 * nq]
    np.testing.assert_allclose(proj, dq, rtol=1e-9)
    # gamma = 0 is the observed step (to the rounding of f^eq(v) - f^eq(v))
    zero = Simulation(wl, u0, gamma_fixed=np.zeros(nq))
    zero.run(1)
    np.testing.assert_allclose(zero.fp, obs.fp, rtol=0, atol=1e-15)


def test_mean_profile_sum_on_a_laminar_channel():
    """The running mean-profile sum (the <u_x>(y) statistic of Sec. 7.3) on the
    body-force channel at tau = 1/2 + sqrt(3)/4, where the steady profile is
    exactly the parabola F y_w (2H - y_w)/(2 nu) (Poiseuille, pinned above):
    the stored post-collision velocity is that physical velocity plus
    F/(2 rho), so K steps add K (parabola + F/2) on every fluid row and zero
    on the solid rows.  A perturbation a (-1)^x cos(pi z/2) of zero plane mean
    (a = 1e-9) leaves the plane mean unchanged to O(a^2), so the sum must
    average over the whole x-z plane, not one column."""
    fx, ny, nx, nz = 1e-6, 10, 4, 4
    tau = 0.5 + math.sqrt(3) / 4
    base = synthetic.workload("C3", nx=nx, ny=ny, nz=nz, tau=tau, forcing="guo", body_force=(fx, 0.0, 0.0),
                              substrate="none", to_mode="off", init=("rest",), n_mp=0)
    spin = Simulation(base, np.zeros((3, nz, ny, nx)))
    spin.run(2500)
    lat = spin.lat
    rho, v = spin.macros()
    x = np.arange(nx)[None, None, :]
    z = np.arange(nz)[:, None, None]
    pert = 1e-9 * ((-1.0) ** x) * np.cos(np.pi * z / 2) * spin.mask
    v2 = v.copy()
    v2[0] += pert
    fp = spin.fp + lbm.equilibrium(lat, rho, v2) - lbm.equilibrium(lat, rho, v)
    obs = Simulation(dict(base, to_mode="observe", qois=[("E", "B", 1)], h=0), np.zeros((3, nz, ny, nx)))
    obs.fp = fp
    k = 4
    obs.run(k)
    nu = CS2 * (tau - 0.5)
    yw = np.arange(ny) - 0.5
    exact = fx / (2 * nu) * yw * ((ny - 2) - yw) + 0.5 * fx
    exact[0] = exact[-1] = 0.0
    np.testing.assert_allclose(obs.profile_sum / k, exact, rtol=1e-9, atol=1e-20)
