"""ctypes binding of liblbm.so (include/lbm.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  There is no fallback: if liblbm.so is missing or fails to load,
importing this module raises.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_BUDGET, LBM_ERR_CUDA, LBM_ERR_UNSTABLE = 0, 1, 2, 3, 4
LBM_ERR_SINGULAR_GRAM, LBM_ERR_TIMEOUT, LBM_ERR_STATE = 5, 6, 7
FORCING = {"edm": 0, "guo": 1}
SUBSTRATE = {"none": 0, "smag": 1, "wale": 2}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
QOI_KIND = {"E": 0, "Z": 1}
FILTER = {"G": 0, "L": 1, "B": 2, "F": 3}
TO_MODE = {"off": 0, "observe": 1, "gamma": 2, "lrs": 3, "track": 4, "fixed": 5}
MAX_QOI = 16
FLAG_SINGULAR, FLAG_UNSTABLE = 1, 2
# profile classes, in the order of the LBM_K_* ids of include/lbm.h
K_NAMES = ["predict", "collide", "curl", "filter", "sens", "reduce", "lrs", "solve", "apply", "gauss_x", "lap1", "fft",
           "wale", "gauss_z", "gauss_y", "lap3", "reserved16", "totals"]
EXPORTED = [
    "lbm_qoi_row_len", "lbm_required_bytes", "lbm_create", "lbm_destroy", "lbm_last_error", "lbm_init_macros",
    "lbm_set_lrs", "lbm_set_to_coeffs", "lbm_set_track_reference", "lbm_step", "lbm_sync", "lbm_qoi", "lbm_get_macros",
    "lbm_get_populations", "lbm_set_populations", "lbm_get_profile", "lbm_get_step", "lbm_state_bytes",
    "lbm_save", "lbm_load", "lbm_set_graphs", "lbm_profile", "lbm_profile_read", "lbm_launches_per_step",
    "lbm_qoi_eval_static", "lbm_filter_flops_per_step",
    "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_admit", "lbm_batch_member", "lbm_batch_run",
    "lbm_batch_poll", "lbm_batch_release", "lbm_batch_stats", "lbm_set_autotune", "lbm_get_tuning", "lbm_set_branching",
    "lbm_project_shape", "lbm_project", "lbm_eval_qoi", "lbm_set_launch_goal", "lbm_batch_wait",
    "lbm_batch_set_persistent",
]


class lbm_completion(C.Structure):
    _fields_ = [("slot", C.c_int32), ("status", C.c_int32), ("steps", C.c_int64), ("tag", C.c_uint64),
                ("t_done_ms", C.c_double)]


class lbm_qoi_spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("filter", C.c_int32), ("scale", C.c_int32), ("band_hi", C.c_int32)]


class lbm_config(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("walls", C.c_int32), ("forcing", C.c_int32), ("substrate", C.c_int32), ("storage", C.c_int32),
        ("tau", C.c_double), ("body_force", C.c_double * 3), ("kolmo_amp", C.c_double),
        ("kolmo_drag", C.c_double), ("kolmo_k", C.c_int32), ("to_mode", C.c_int32),
        ("c_smag", C.c_double), ("c_wale", C.c_double), ("n_qoi", C.c_int32), ("n_mp", C.c_int32),
        ("qoi", lbm_qoi_spec * MAX_QOI), ("h", C.c_int32), ("qoi_ring", C.c_int32),
        ("gamma_std", C.c_double), ("seed", C.c_uint64), ("member", C.c_uint64), ("track_len", C.c_int64),
        ("spinup", C.c_int64),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblbm.so not built ({LIB_PATH}); run python -m paper_2609_32892_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, VP, I64, PI64, PD = C.POINTER, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    cfg = P(lbm_config)
    sig = {
        "lbm_qoi_row_len": [cfg, PI64],
        "lbm_required_bytes": [cfg, P(C.c_size_t)],
        "lbm_create": [cfg, VP, C.c_size_t, VP, P(VP)],
        "lbm_destroy": [VP],
        "lbm_last_error": [VP, C.c_char_p, C.c_size_t],
        "lbm_init_macros": [VP, PD, PD],
        "lbm_set_lrs": [VP, PD, PD, PD, PD, PD, PD],
        "lbm_set_to_coeffs": [VP, C.c_int, C.c_int32, PD, PD, PD, PD, PD],
        "lbm_set_track_reference": [VP, PD, I64],
        "lbm_step": [VP, I64],
        "lbm_sync": [VP],
        "lbm_qoi": [VP, PD, I64, PI64, PI64],
        "lbm_get_macros": [VP, PD, PD],
        "lbm_get_populations": [VP, PD],
        "lbm_set_populations": [VP, PD],
        "lbm_get_profile": [VP, PD, PI64],
        "lbm_get_step": [VP, PI64],
        "lbm_state_bytes": [VP, P(C.c_size_t)],
        "lbm_save": [VP, VP, C.c_size_t],
        "lbm_load": [VP, VP, C.c_size_t],
        "lbm_set_graphs": [VP, C.c_int],
        "lbm_profile": [VP, C.c_int],
        "lbm_profile_read": [VP, PD, PI64, C.c_int],
        "lbm_launches_per_step": [VP, PI64],
        "lbm_qoi_eval_static": [cfg, VP, VP, VP],
        "lbm_filter_flops_per_step": [VP, PD, C.c_int],
        "lbm_batch_create": [C.c_int32, VP, C.c_size_t, P(VP)],
        "lbm_batch_destroy": [VP],
        "lbm_batch_admit": [VP, cfg, PD, I64, C.c_uint64, P(C.c_int32)],
        "lbm_batch_member": [VP, C.c_int32, P(VP)],
        "lbm_batch_run": [VP, I64],
        "lbm_batch_poll": [VP, P(lbm_completion), C.c_int32, P(C.c_int32)],
        "lbm_batch_release": [VP, C.c_int32],
        "lbm_batch_stats": [VP, P(C.c_size_t), P(C.c_size_t), P(C.c_int32)],
        "lbm_set_autotune": [VP, C.c_int],
        "lbm_set_branching": [VP, C.c_int],
        "lbm_set_launch_goal": [VP, C.c_int],
        "lbm_batch_wait": [VP, C.c_int32],
        "lbm_batch_set_persistent": [VP, C.c_int, I64],
        "lbm_project_shape": [C.POINTER(lbm_config), C.c_int, C.POINTER(C.c_int32)],
        "lbm_project": [VP, C.c_int, VP, VP],
        "lbm_eval_qoi": [VP, VP, VP],
        "lbm_get_tuning": [VP, P(C.c_int32), C.c_int],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    return lib


_lib = _load()


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm status {code}: {msg}")
        self.code = code


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def last_error(ctx=None):
    buf = C.create_string_buffer(256)
    _lib.lbm_last_error(ctx, buf, 256)
    return buf.value.decode()


def _check(rc, ctx=None):
    if rc != LBM_OK:
        raise LbmError(rc, last_error(ctx))


# ---------------------------------------------------------------- configs --
def config_from_workload(wl, member=0):
    """lbm_config of a workload dict (see synthetic.workloads)."""
    c = lbm_config()
    c.dim, c.nx, c.ny, c.nz = wl["dim"], wl["nx"], wl["ny"], wl["nz"]
    c.walls = 1 if wl["walls"] else 0
    c.forcing = FORCING[wl["forcing"]]
    c.substrate = SUBSTRATE[wl["substrate"]]
    c.storage = STORAGE[wl.get("storage", "fp32")]
    c.tau = wl["tau"]
    for a in range(3):
        c.body_force[a] = wl["body_force"][a]
    c.kolmo_amp, c.kolmo_drag, c.kolmo_k = wl["kolmo_amp"], wl["kolmo_drag"], wl["kolmo_k"]
    c.to_mode = TO_MODE[wl["to_mode"]]
    c.c_smag, c.c_wale = wl["c_smag"], wl["c_wale"]
    qois = wl["qois"] if wl["to_mode"] != "off" else []
    c.n_qoi = len(qois)
    c.n_mp = wl["n_mp"] if wl["to_mode"] != "off" else 0
    for i, (kind, filt, scale) in enumerate(qois):
        c.qoi[i].kind, c.qoi[i].filter = QOI_KIND[kind], FILTER[filt]
        if filt == "F":
            c.qoi[i].scale, c.qoi[i].band_hi = scale
        else:
            c.qoi[i].scale = scale
    c.h = wl["h"]
    c.qoi_ring = wl.get("qoi_ring", 0)
    c.gamma_std = wl["gamma_std"]
    c.seed = wl["seed"]
    c.member = member
    c.track_len = wl.get("track_len", 0)
    c.spinup = wl.get("spinup", 0)
    return c


# ------------------------------------------------------------ C-ABI calls --
def lbm_qoi_row_len(cfg):
    n = C.c_int64()
    _check(_lib.lbm_qoi_row_len(C.byref(cfg), C.byref(n)))
    return n.value


def lbm_required_bytes(cfg):
    n = C.c_size_t()
    _check(_lib.lbm_required_bytes(C.byref(cfg), C.byref(n)))
    return n.value


def lbm_create(cfg, dev_ptr, nbytes, stream_ptr):
    h = C.c_void_p()
    _check(_lib.lbm_create(C.byref(cfg), C.c_void_p(dev_ptr), nbytes, C.c_void_p(stream_ptr), C.byref(h)))
    return h


def lbm_destroy(ctx):
    _check(_lib.lbm_destroy(ctx))


def lbm_init_macros(ctx, rho, u):
    rho, u = _f64(rho), _f64(u)
    _check(_lib.lbm_init_macros(ctx, _ptr(rho), _ptr(u)), ctx)


def lbm_set_lrs(ctx, c_mat, mu, sigma, sigma_ref, q_hist=None, qs_hist=None):
    a = [_f64(x) for x in (c_mat, mu, sigma, sigma_ref, q_hist, qs_hist)]
    _check(_lib.lbm_set_lrs(ctx, *[_ptr(x) for x in a]), ctx)


def lbm_set_to_coeffs(ctx, mode, h=0, c_mat=None, mu=None, sigma=None, sigma_ref=None, gamma_fixed=None):
    """mode: a TO_MODE name or value (must be the context's configured mode)."""
    m = TO_MODE[mode] if isinstance(mode, str) else int(mode)
    a = [_f64(x) for x in (c_mat, mu, sigma, sigma_ref, gamma_fixed)]
    _check(_lib.lbm_set_to_coeffs(ctx, m, int(h), *[_ptr(x) for x in a]), ctx)


def lbm_set_track_reference(ctx, qref):
    q = _f64(qref)
    _check(_lib.lbm_set_track_reference(ctx, _ptr(q), q.shape[0]), ctx)


def lbm_step(ctx, nsteps):
    _check(_lib.lbm_step(ctx, int(nsteps)), ctx)


def lbm_sync(ctx):
    _check(_lib.lbm_sync(ctx), ctx)


def lbm_qoi(ctx, row_len, capacity=65536):
    out = np.zeros((capacity, row_len))
    nw, nl = C.c_int64(), C.c_int64()
    _check(_lib.lbm_qoi(ctx, _ptr(out), capacity, C.byref(nw), C.byref(nl)), ctx)
    return out[: nw.value], nl.value


def lbm_get_macros(ctx, shape_zyx):
    nz, ny, nx = shape_zyx
    rho = np.zeros((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    _check(_lib.lbm_get_macros(ctx, _ptr(rho), _ptr(u)), ctx)
    return rho, u


def lbm_get_populations(ctx, q, shape_zyx):
    f = np.zeros((q,) + tuple(shape_zyx))
    _check(_lib.lbm_get_populations(ctx, _ptr(f)), ctx)
    return f


def lbm_set_populations(ctx, f):
    f = _f64(f)
    _check(_lib.lbm_set_populations(ctx, _ptr(f)), ctx)


def lbm_get_profile(ctx, ny):
    prof = np.zeros(ny)
    n = C.c_int64()
    _check(_lib.lbm_get_profile(ctx, _ptr(prof), C.byref(n)), ctx)
    return prof, n.value


def lbm_get_step(ctx):
    n = C.c_int64()
    _check(_lib.lbm_get_step(ctx, C.byref(n)), ctx)
    return n.value


def lbm_state_bytes(ctx):
    n = C.c_size_t()
    _check(_lib.lbm_state_bytes(ctx, C.byref(n)), ctx)
    return n.value


def lbm_save(ctx):
    n = lbm_state_bytes(ctx)
    buf = (C.c_char * n)()
    _check(_lib.lbm_save(ctx, C.cast(buf, C.c_void_p), n), ctx)
    return bytes(buf)


def lbm_load(ctx, blob):
    buf = C.create_string_buffer(blob, len(blob))
    _check(_lib.lbm_load(ctx, C.cast(buf, C.c_void_p), len(blob)), ctx)


def lbm_set_graphs(ctx, enable):
    _check(_lib.lbm_set_graphs(ctx, int(bool(enable))), ctx)


def lbm_profile(ctx, enable):
    _check(_lib.lbm_profile(ctx, int(bool(enable))), ctx)


def lbm_profile_read(ctx):
    ms = np.zeros(len(K_NAMES))
    n = np.zeros(len(K_NAMES), dtype=np.int64)
    _check(_lib.lbm_profile_read(ctx, _ptr(ms), n.ctypes.data_as(C.POINTER(C.c_int64)), len(K_NAMES)), ctx)
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(K_NAMES)}


def lbm_filter_flops_per_step(ctx):
    f = np.zeros(len(K_NAMES))
    _check(_lib.lbm_filter_flops_per_step(ctx, _ptr(f), len(K_NAMES)), ctx)
    return {k: float(f[i]) for i, k in enumerate(K_NAMES)}


def lbm_launches_per_step(ctx):
    n = C.c_int64()
    _check(_lib.lbm_launches_per_step(ctx, C.byref(n)), ctx)
    return n.value


def lbm_qoi_eval_static(cfg, u_dev_ptr, q_dev_ptr, stream_ptr):
    """Scale-aware QoIs of a device velocity field using only the library's
    built-in scratch array (for callers that cannot allocate device memory)."""
    _check(_lib.lbm_qoi_eval_static(C.byref(cfg), C.c_void_p(u_dev_ptr), C.c_void_p(q_dev_ptr),
                                    C.c_void_p(stream_ptr)))


# ---------------------------------------------------------------- batches --
def lbm_batch_create(n_slots, pool_ptr, pool_bytes):
    h = C.c_void_p()
    _check(_lib.lbm_batch_create(int(n_slots), C.c_void_p(pool_ptr), pool_bytes, C.byref(h)))
    return h


def lbm_batch_destroy(b):
    _check(_lib.lbm_batch_destroy(b))


def lbm_batch_admit(b, cfg, u0, horizon, tag=0):
    """Admit a member; returns its slot, or None when it does not fit (LBM_ERR_BUDGET)."""
    u = _f64(u0)
    s = C.c_int32()
    rc = _lib.lbm_batch_admit(b, C.byref(cfg), _ptr(u), int(horizon), int(tag), C.byref(s))
    if rc == LBM_ERR_BUDGET:
        return None
    _check(rc)
    return s.value


def lbm_batch_member(b, slot):
    h = C.c_void_p()
    _check(_lib.lbm_batch_member(b, int(slot), C.byref(h)))
    return h


def lbm_batch_run(b, steps):
    _check(_lib.lbm_batch_run(b, int(steps)))


def lbm_batch_set_persistent(b, lanes, max_nodes=16384):
    """lanes: 0 = per-member graphs for every member; n > 0 = persistent batched
    kernels (n lanes per class) for members of at most max_nodes nodes."""
    _check(_lib.lbm_batch_set_persistent(b, int(lanes), int(max_nodes)))


def lbm_batch_wait(b, rounds):
    _check(_lib.lbm_batch_wait(b, int(rounds)))


def lbm_batch_poll(b, cap=256):
    arr = (lbm_completion * cap)()
    n = C.c_int32()
    _check(_lib.lbm_batch_poll(b, arr, cap, C.byref(n)))
    return [dict(slot=arr[i].slot, status=arr[i].status, steps=arr[i].steps, tag=arr[i].tag,
                 t_done_ms=arr[i].t_done_ms) for i in range(n.value)]


def lbm_batch_release(b, slot):
    _check(_lib.lbm_batch_release(b, int(slot)))


def lbm_batch_stats(b):
    f, l, a = C.c_size_t(), C.c_size_t(), C.c_int32()
    _check(_lib.lbm_batch_stats(b, C.byref(f), C.byref(l), C.byref(a)))
    return f.value, l.value, a.value


def lbm_set_autotune(ctx, enable):
    _check(_lib.lbm_set_autotune(ctx, int(bool(enable))), ctx)


def lbm_set_branching(ctx, enable):
    _check(_lib.lbm_set_branching(ctx, int(bool(enable))), ctx)


GOAL_LATENCY, GOAL_THROUGHPUT = 0, 1


def lbm_set_launch_goal(ctx, goal):
    _check(_lib.lbm_set_launch_goal(ctx, int(goal)), ctx)


def lbm_project_shape(cfg, m):
    """LF grid (nx, ny, nz) of the projection phi_m of a configuration."""
    d = (C.c_int32 * 3)()
    _check(_lib.lbm_project_shape(C.byref(cfg), int(m), d), None)
    return tuple(int(v) for v in d)


def lbm_project(ctx, m, drho_ptr, u_ptr):
    """Enqueue phi_m of the context's state into device buffers (raw pointers)."""
    _check(_lib.lbm_project(ctx, int(m), C.c_void_p(drho_ptr), C.c_void_p(u_ptr)), ctx)


def lbm_eval_qoi(ctx, u_ptr, q_ptr):
    """Enqueue the context's QoIs of a device velocity field into a device array."""
    _check(_lib.lbm_eval_qoi(ctx, C.c_void_p(u_ptr), C.c_void_p(q_ptr)), ctx)


def lbm_get_tuning(ctx):
    v = (C.c_int32 * 14)()
    _check(_lib.lbm_get_tuning(ctx, v, 14), ctx)
    return {"tuned": int(v[0]), "collide_pair": int(v[1]), "corrector_in_collide": int(v[2]), "march_threads": int(v[3]),
            "filter_blocks_per_sm": [int(v[4 + f]) for f in range(8)], "throughput_goal": int(v[12]),
            "predict_pair": int(v[13])}
