"""Workload descriptions: the paper's two flows at the benchmark sizes.

A workload is a plain dict of parameters.  Keys:

  dim, nx, ny, nz     lattice (2-D: nz = 1; D2Q9 in 2-D, D3Q19 in 3-D)
  walls               halfway bounce-back walls in y (rows 0 and ny-1 solid)
  tau                 BGK relaxation time
  forcing             'edm' (exact difference method) or 'guo'
  body_force          constant force density (Fx, Fy, Fz)
  kolmo_amp, kolmo_k  Kolmogorov force density amp*sin(2*pi*k*y/ny) along x
  kolmo_drag          linear drag rate alpha: force density -alpha * rho v
  substrate           'none' | 'smag' | 'wale', with c_smag / c_wale
  qois                list of (kind, filter, scale): kind 'E' or 'Z',
                      filter 'G' (Gaussian), 'L' (Laplacian), 'B' (3x3 binomial)
                      or 'F' (sharp Fourier band, scale = (l, m) wavenumber bins)
  n_mp                number of mean-profile QoIs (channel only)
  to_mode             'off' | 'observe' | 'gamma' | 'fixed' | 'lrs' | 'track'
                      ('fixed': the caller's gamma_i held for every step)
  gamma_std           std of the per-step random gamma ('gamma' mode)
  h                   LRS history length
  seed                run seed (Philox key and input generators)
  init                ('noise', amp) or ('channel', u_c, noise_frac)
  storage             'fp32' | 'fp16' | 'bf16' (GPU population storage)
  steps               steps of the full run
"""

import copy
import math

from .units import channel_lattice, kolmogorov_lattice

SCALE_QOIS_3D = [("E", "G", 3), ("Z", "G", 3), ("E", "L", 3), ("Z", "L", 3), ("E", "L", 1), ("Z", "L", 1)]


def _base():
    return dict(dim=2, nx=8, ny=8, nz=1, walls=False, tau=0.6, forcing="edm", body_force=(0.0, 0.0, 0.0),
                kolmo_amp=0.0, kolmo_k=0, kolmo_drag=0.0, substrate="none", c_smag=0.1, c_wale=0.5,
                qois=[], n_mp=0, to_mode="off", gamma_std=0.0, h=0, seed=1234, init=("noise", 1e-3),
                storage="fp32", steps=10)


def _c1():
    w = _base()
    w.update(name="kolmogorov2d_64_fp64_gamma", dim=2, nx=64, ny=64, tau=0.52, forcing="guo",
             kolmo_amp=1e-5, kolmo_k=4, qois=[("E", "B", 1), ("Z", "B", 1)], to_mode="gamma",
             gamma_std=1e-2, seed=20260901, init=("noise", 1e-3), steps=2000)
    return w


def _c2():
    p = kolmogorov_lattice(256)
    w = _base()
    w.update(name="kolmogorov2d_256_smag_tolrs", dim=2, nx=256, ny=256, tau=p["tau"], forcing="guo",
             kolmo_amp=p["kolmo_amp"], kolmo_k=4, kolmo_drag=p["kolmo_drag"], substrate="smag", c_smag=0.1,
             qois=[("E", "G", 3), ("Z", "G", 3), ("E", "L", 1), ("Z", "L", 1)], to_mode="lrs", h=400,
             seed=20260902, init=("noise", 1e-3), steps=20000)
    return w


def _c3():
    p = channel_lattice(40)
    w = _base()
    w.update(name="channel3d_96x40x48_wale_tolrs", dim=3, nx=96, ny=40, nz=48, walls=True, tau=p["tau"],
             forcing="edm", body_force=(p["body_force"], 0.0, 0.0), substrate="wale", c_wale=2.20,
             qois=list(SCALE_QOIS_3D), n_mp=6, to_mode="lrs", h=500, seed=20260903,
             init=("channel", 0.1, 0.05), steps=50000)
    return w


def _c4():
    p = channel_lattice(200)
    w = _base()
    w.update(name="channel3d_480x200x240_bgk", dim=3, nx=480, ny=200, nz=240, walls=True, tau=p["tau"],
             forcing="edm", body_force=(p["body_force"], 0.0, 0.0), seed=20260904,
             init=("channel", 0.1, 0.05), steps=2000)
    return w


def _c4_to():
    """The full TO-LRS channel step (C3 physics) on the 480x200x240 grid."""
    p = channel_lattice(200)
    w = _c3()
    w.update(name="channel3d_480x200x240_wale_tolrs", nx=480, ny=200, nz=240, tau=p["tau"],
             body_force=(p["body_force"], 0.0, 0.0), seed=20260905, steps=2000)
    return w


def _c4_to_mid():
    """The TO-LRS channel step on a 320x200x160 grid (10.2 M nodes): fields larger
    than L2 but a few GB on the device, for profiler captures."""
    w = _c4_to()
    w.update(name="channel3d_320x200x160_wale_tolrs", nx=320, nz=160, seed=20260906)
    return w


def _c2f():
    """The Kolmogorov LES with sharp Fourier-band QoIs (App. E bins on 128^2)."""
    p = kolmogorov_lattice(128)
    w = _c2()
    w.update(name="kolmogorov2d_128_smag_tolrs_fourier", nx=128, ny=128, tau=p["tau"], kolmo_amp=p["kolmo_amp"],
             kolmo_drag=p["kolmo_drag"],
             qois=[("E", "F", (0, 12)), ("Z", "F", (0, 12)), ("E", "F", (13, 32)), ("Z", "F", (13, 32)),
                   ("E", "F", (33, 128)), ("Z", "F", (33, 128))], seed=20260907)
    return w


def _hf_channel():
    """HF reference run of Sec. 7.1: plain BGK channel on the 1475x237x490 grid
    (171 M nodes), projected by phi_5 onto the 295x49x98 LF grid."""
    p = channel_lattice(237)
    w = _base()
    w.update(name="channel3d_1475x237x490_bgk_hf", dim=3, nx=1475, ny=237, nz=490, walls=True, tau=p["tau"],
             forcing="edm", body_force=(p["body_force"], 0.0, 0.0), seed=20260908,
             init=("channel", 0.1, 0.05), steps=2000)
    return w


def _hf_channel_480():
    """HF reference run at the 480x200x240 benchmark scale: plain BGK channel on
    480x192x240 (22.1 M nodes), projected by phi_5 onto C3's 96x40x48 grid."""
    p = channel_lattice(192)
    w = _hf_channel()
    w.update(name="channel3d_480x192x240_bgk_hf", nx=480, ny=192, nz=240, tau=p["tau"],
             body_force=(p["body_force"], 0.0, 0.0), seed=20260911)
    return w


def _lf_channel():
    """The LF channel LES of Sec. 7.1 (295x49x98, WALE + TO-LRS, 12 QoIs): the
    grid phi_5 of the HF run lands on."""
    p = channel_lattice(49)
    w = _c3()
    w.update(name="channel3d_295x49x98_wale_tolrs", nx=295, ny=49, nz=98, tau=p["tau"],
             body_force=(p["body_force"], 0.0, 0.0), seed=20260909)
    return w


def _hf_kolmo():
    """HF reference run of Sec. 6: plain BGK Kolmogorov flow on 2048^2,
    projected by phi_8 (bicubic) onto the 256^2 LF grid of C2."""
    p = kolmogorov_lattice(2048)
    w = _base()
    w.update(name="kolmogorov2d_2048_bgk_hf", dim=2, nx=2048, ny=2048, tau=p["tau"], forcing="guo",
             kolmo_amp=p["kolmo_amp"], kolmo_k=4, kolmo_drag=p["kolmo_drag"], seed=20260910,
             init=("noise", 1e-3), steps=20000)
    return w


WORKLOADS = {
    "HF_CHANNEL": _hf_channel,
    "HF_CHANNEL_480": _hf_channel_480,
    "LF_CHANNEL": _lf_channel,
    "HF_KOLMO": _hf_kolmo,
    "C1": _c1,
    "C2": _c2,
    "C3": _c3,
    "C4": _c4,
    "C4_TO": _c4_to,
    "C4_TO_MID": _c4_to_mid,
    "C2F": _c2f,
}


def workload(name, **overrides):
    """A fresh copy of a named workload with keyword overrides applied."""
    w = copy.deepcopy(WORKLOADS[name]())
    w.update(overrides)
    return w


def serving_mix(n_members, seed, rate_per_s):
    """Poisson request stream of mixed 2-D/3-D ensemble members.

    Sizes are uniform over {128, 256, 384, 512}^2 (Kolmogorov, Smagorinsky +
    TO-LRS with 4 QoIs) and {48x20x24, 72x30x36, 96x40x48} (channel, WALE +
    TO-LRS with 12 QoIs); horizons are log-uniform in [1e3, 1e4] steps.
    """
    import numpy as np

    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    sizes2 = [128, 256, 384, 512]
    sizes3 = [(48, 20, 24), (72, 30, 36), (96, 40, 48)]
    for m in range(n_members):
        t += rng.exponential(1.0 / rate_per_s)
        if rng.uniform() < 0.5:
            n = int(sizes2[rng.integers(len(sizes2))])
            p = kolmogorov_lattice(n)
            w = _c2()
            w.update(nx=n, ny=n, tau=p["tau"], kolmo_amp=p["kolmo_amp"], kolmo_drag=p["kolmo_drag"])
        else:
            nx, ny, nz = sizes3[rng.integers(len(sizes3))]
            p = channel_lattice(ny)
            w = _c3()
            w.update(nx=nx, ny=ny, nz=nz, tau=p["tau"], body_force=(p["body_force"], 0.0, 0.0))
        w["seed"] = int(seed * 1000 + m)
        w["steps"] = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e4)))))
        w["arrival_s"] = t
        w["name"] = f"member{m}"
        out.append(w)
    return out


def serving_requests(n_members, seed, rate_per_s, horizon_scale=1.0, storage="fp32"):
    """The serving mix as server requests: each member's workload with its
    seeded initial field (u0), its synthetic LRS model (lrs: C, mu, Sigma and
    sigma_ref = 0, i.e. scales from the member's first step), its steps per
    simulated time unit, horizons scaled by horizon_scale and the population
    storage precision."""
    import math

    from .fields import initial_velocity
    from .lrs_inputs import synthetic_lrs

    reqs = serving_mix(n_members, seed, rate_per_s)
    for r in reqs:
        r["steps"] = max(2, int(math.ceil(r["steps"] * horizon_scale)))
        r["storage"] = storage
        r["u0"] = initial_velocity(r)
        nq = len(r["qois"]) + r["n_mp"]
        c, mu, sig = synthetic_lrs(nq, r["h"], r["seed"])
        r["lrs"] = (c, mu, sig, [0.0] * nq)
        lat = kolmogorov_lattice(r["nx"]) if r["dim"] == 2 else channel_lattice(r["ny"])
        r["steps_per_tu"] = lat["steps_per_tu"]
    return reqs
