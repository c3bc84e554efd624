"""Pins for the projection phi_m (Sec. 3) and the HF reference series.

The bicubic projection is pinned by the interpolation property, the
textbook four-point midpoint rule and exact cubic reproduction at
half-spacing offsets, and a direct 16-term evaluation; the wall-anchored
subsampling by the grid and wall-unit figures of Sec. 7.1 and by the wall
distances it must preserve.
"""

import json
import os

import numpy as np
import pytest

import synthetic
from oracle import projection as P
from oracle.sim import Simulation
from oracle.to import TOSetup

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_keys_kernel_interpolates_and_sums_to_one():
    assert P.keys_kernel(0.0) == 1.0
    for t in (1.0, -1.0, 2.0, -2.0, 2.5, -3.0):
        assert P.keys_kernel(t) == 0.0
    for t in np.linspace(0.0, 1.0, 17, endpoint=False):
        w = [P.keys_kernel(t - k) for k in (-1, 0, 1, 2)]
        assert abs(sum(w) - 1.0) < 1e-15
    # half-way between nodes: the four-point cubic midpoint rule (-1, 9, 9, -1)/16
    w = [float(P.keys_kernel(0.5 - k)) for k in (-1, 0, 1, 2)]
    assert w == [-1 / 16, 9 / 16, 9 / 16, -1 / 16]


@pytest.mark.parametrize("m", [1, 3, 5])
def test_bicubic_odd_m_is_block_centre_subsampling(m):
    rng = np.random.default_rng(m)
    a = rng.standard_normal((2, 4 * m, 6 * m))
    c = (m - 1) // 2
    np.testing.assert_array_equal(P.project_bicubic_2d(a, m), a[:, c::m, c::m])


@pytest.mark.parametrize("m", [2, 4, 8])
def test_bicubic_even_m_reproduces_cubics(m):
    """At half-spacing offsets the Keys weights are cubic Lagrange weights:
    a separable bicubic polynomial is reproduced exactly where the stencil
    does not wrap."""
    n = 6 * m
    x = np.arange(n, dtype=np.float64)
    px = 0.3 - 0.7 * x + 0.05 * x**2 - 0.002 * x**3
    py = 1.1 + 0.2 * x - 0.01 * x**2 + 0.0007 * x**3
    a = np.outer(py, px)  # [y, x]
    out = P.project_bicubic_2d(a, m)
    X = m * np.arange(n // m) + 0.5 * (m - 1)
    ok = (np.floor(X) - 1 >= 0) & (np.floor(X) + 2 <= n - 1)
    fx = 0.3 - 0.7 * X + 0.05 * X**2 - 0.002 * X**3
    fy = 1.1 + 0.2 * X - 0.01 * X**2 + 0.0007 * X**3
    want = np.outer(fy, fx)
    np.testing.assert_allclose(out[np.ix_(ok, ok)], want[np.ix_(ok, ok)], rtol=1e-12, atol=1e-12)


def test_bicubic_matches_direct_sixteen_point_sum():
    m, ny, nx = 4, 12, 16
    rng = np.random.default_rng(7)
    a = rng.standard_normal((ny, nx))
    out = P.project_bicubic_2d(a, m)

    def w(t):  # Keys a = -1/2, written out independently
        t = abs(t)
        if t <= 1:
            return 1.5 * t**3 - 2.5 * t**2 + 1
        if t < 2:
            return -0.5 * t**3 + 2.5 * t**2 - 4 * t + 2
        return 0.0

    for j, i in [(0, 0), (1, 2), (2, 3), (0, 3)]:
        X, Y = m * i + 1.5, m * j + 1.5
        s = 0.0
        for yy in range(-3, ny + 3):
            for xx in range(-3, nx + 3):
                s += w(X - xx) * w(Y - yy) * a[yy % ny, xx % nx]
        assert abs(out[j, i] - s) < 1e-13


def test_bicubic_constant_and_smooth_mode():
    m, n = 8, 64
    np.testing.assert_allclose(P.project_bicubic_2d(np.full((n, n), 2.5), m), 2.5, rtol=0, atol=1e-15)
    x = np.arange(n)
    a = np.sin(2 * np.pi * x / n)[None, :] * np.ones((n, 1))
    X = m * np.arange(n // m) + 0.5 * (m - 1)
    err = np.abs(P.project_bicubic_2d(a, m) - np.sin(2 * np.pi * X / n)[None, :]).max()
    h = 2 * np.pi / n
    assert err < h**3  # cubic convolution is third-order accurate


def test_anchored_grid_of_the_channel_case():
    g = GOLDEN["channel_projection"]
    assert P.lf_shape_3d(*g["hf"], g["m"]) == tuple(g["lf"])
    rows = P.anchored_rows(g["hf"][1], g["m"])
    assert rows[0] == 0 and rows[-1] == g["hf"][1] - 1
    # walls coincide: LF fluid row j sits m times farther from each wall
    ny_h, ny_l, m = g["hf"][1], g["lf"][1], g["m"]
    for j in range(1, ny_l - 1):
        assert rows[j] - 0.5 == m * (j - 0.5)
        assert (ny_h - 1.5) - rows[j] == m * ((ny_l - 1.5) - j)
    # first fluid nodes in wall units (HF 0.77, LF 3.8, spacings 1.53 and 7.7)
    dp_hf = g["dplus_hf"]
    assert abs((rows[1] - 0.5) * dp_hf - g["yplus_lf_first"]) < 0.05
    assert abs(0.5 * dp_hf - g["yplus_hf_first"]) < 0.01
    assert abs(m * dp_hf - g["dplus_lf"]) < 0.05


def test_stride_projection_samples_the_anchored_nodes():
    m, nx, ny, nz = 3, 12, 2 + 3 * 4, 9
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, nz, ny, nx))
    out = P.project_stride_3d(a, m)
    assert out.shape == (2, nz // m, 6, nx // m)
    for k in range(nz // m):
        for j in range(6):
            for i in range(nx // m):
                yh = 0 if j == 0 else (ny - 1 if j == 5 else m * j - 1)
                assert out[1, k, j, i] == a[1, m * k + 1, yh, m * i + 1]


def test_projection_rejects_bad_sizes():
    with pytest.raises(ValueError):
        P.lf_shape_3d(20, 22, 20, 4)  # even m
    with pytest.raises(ValueError):
        P.lf_shape_3d(20, 23, 20, 5)  # ny - 2 not divisible
    with pytest.raises(ValueError):
        P.project_bicubic_2d(np.zeros((10, 12)), 4)


@pytest.mark.parametrize("name,kw", [("C2", dict(nx=24, ny=24)), ("C3", dict(nx=12, ny=14, nz=9))])
def test_reference_with_m1_equals_observed_qois(name, kw):
    """With m = 1 the reference series is the run's own QoI series: the
    projection path (macros, phi_1, Q) agrees with the QoIs an observing run
    takes inside its step."""
    wl = synthetic.workload(name, to_mode="observe", **kw)
    obs = Simulation(wl, synthetic.initial_velocity(wl))
    rows = obs.run(4)
    hf = Simulation(dict(wl, to_mode="off"), synthetic.initial_velocity(wl))
    setup = TOSetup(wl["dim"], wl["nx"], wl["ny"], wl["nz"], wl["walls"], wl["qois"], wl["n_mp"])
    ref = P.hf_reference(hf, setup, 1, 4)
    nq = setup.nq
    np.testing.assert_allclose(ref, rows[:, 1:1 + nq], rtol=1e-12, atol=1e-300)
