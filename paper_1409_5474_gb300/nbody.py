"""ctypes binding of libnbody.so (include/nbody.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; the force, predictor, corrector and scheduler run in the
library's CUDA kernels. If the library has not been built, ``load()`` raises:
there is no CPU fallback.

Array conventions follow the C ABI: a vector field over n particles is a
(3, n) float64 array (rows x, y, z); masses, potentials, times and steps are
(n,) float64 arrays; indices are int32. Host-array calls copy in and out;
``nb_force_dev`` takes device pointers (e.g. ``tensor.data_ptr()``) and runs
on the handle's stream (``nb_set_stream``, e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbody.so")

NB_OK = 0
NB_ERR_ARG = 1
NB_ERR_OOM = 2
NB_ERR_BUDGET = 3
NB_ERR_CUDA = 4
NB_ERR_TIMEOUT = 5
NB_ERR_NONFINITE = 6
NB_ERR_BUSY = 7
NB_ERR_NOTFOUND = 8
NB_ERR_STATE = 9

NB_F32 = 0
NB_F32DS = 1
NB_F64 = 2
VARIANTS = {"f32": NB_F32, "f32ds": NB_F32DS, "f64": NB_F64}

NB_FLAG_TIMING = 1
NB_FLAG_NO_FUSED = 2
NB_FUSED_MAX_NA = 4096
NB_FUSED_DEFAULT_NA = 1024
NB_FUSED6_MAX_NA = 64
NB_MAX_CORR = 8


class NBodyError(RuntimeError):
    def __init__(self, status, func, msg):
        self.status = status
        self.func = func
        super().__init__(f"{func}: status {status}: {msg}")


class nb_config(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("variant", ctypes.c_int), ("eps", ctypes.c_double),
                ("eta", ctypes.c_double), ("eta_s", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("dt_min", ctypes.c_double), ("shared_dt", ctypes.c_double),
                ("budget_bytes", ctypes.c_size_t), ("device", ctypes.c_int),
                ("flags", ctypes.c_int), ("fused_max_na", ctypes.c_int),
                ("n_corr", ctypes.c_int), ("order", ctypes.c_int)]


class nb_plan(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nwj", ctypes.c_int), ("nsplit", ctypes.c_int)]

    def as_tuple(self):
        return (self.kind, self.nwj, self.nsplit)


class nb_stats(ctypes.Structure):
    _fields_ = [("block_steps", ctypes.c_longlong), ("force_launches", ctypes.c_longlong),
                ("interactions", ctypes.c_double), ("force_ms", ctypes.c_double),
                ("reduce_ms", ctypes.c_double), ("predict_ms", ctypes.c_double),
                ("correct_ms", ctypes.c_double), ("sched_ms", ctypes.c_double),
                ("dt_min_hits", ctypes.c_longlong), ("active_hist", ctypes.c_longlong * 32),
                ("kernel_launches", ctypes.c_longlong),
                ("force_ms_hist", ctypes.c_double * 32), ("inter_hist", ctypes.c_double * 32),
                ("fused_steps", ctypes.c_longlong), ("fused_launches", ctypes.c_longlong),
                ("fused_ms", ctypes.c_double), ("fused_stage_ms", ctypes.c_double * 4),
                ("fused_step_ms_hist", ctypes.c_double * 32)]

    def as_dict(self):
        hists = ("active_hist", "force_ms_hist", "inter_hist", "fused_stage_ms",
                 "fused_step_ms_hist")
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in hists}
        for k in hists:
            d[k] = list(getattr(self, k))
        return d


NB_REQ_FORCE = 0
NB_REQ_EVOLVE = 1
NB_STATUS_QUEUED = 0
NB_STATUS_RUNNING = 1
NB_STATUS_DONE = 2
NB_STATUS_ERROR = 3
NB_STATUS_CANCELLED = 4


class nb_server_cfg(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("variant", ctypes.c_int),
                ("budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("eta", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("flags", ctypes.c_int)]


class nb_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int),
                ("m", ctypes.POINTER(ctypes.c_double)), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("vel", ctypes.POINTER(ctypes.c_double)), ("eps", ctypes.c_double),
                ("t_span", ctypes.c_double)]


class nb_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("error", ctypes.c_int), ("n", ctypes.c_int),
                ("acc", ctypes.POINTER(ctypes.c_double)), ("jerk", ctypes.POINTER(ctypes.c_double)),
                ("pot", ctypes.POINTER(ctypes.c_double)), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("vel", ctypes.POINTER(ctypes.c_double)), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("interactions", ctypes.c_double), ("block_steps", ctypes.c_longlong)]


class nb_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("cancelled", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("ticks", ctypes.c_longlong), ("force_launches", ctypes.c_longlong),
                ("interactions", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("queued", ctypes.c_int), ("inflight", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_H = ctypes.c_void_p
_lib = None
_lock = threading.Lock()

# (name, restype, argtypes); restype int means a status to check
_SIGS = [
    ("nb_config_default", None, [ctypes.POINTER(nb_config)]),
    ("nb_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("nb_last_error", ctypes.c_char_p, [_H]),
    ("nb_version", ctypes.c_char_p, []),
    ("nb_create", ctypes.c_int, [ctypes.POINTER(nb_config), ctypes.POINTER(_H)]),
    ("nb_destroy", ctypes.c_int, [_H]),
    ("nb_set_stream", ctypes.c_int, [_H, ctypes.c_void_p]),
    ("nb_set_particles", ctypes.c_int, [_H, ctypes.c_int, _D, _D, _D, ctypes.c_double]),
    ("nb_init", ctypes.c_int, [_H]),
    ("nb_get_particles", ctypes.c_int, [_H, _D, _D, _D]),
    ("nb_get_state", ctypes.c_int, [_H, _I, _D, _D, _D, _D, _D, _D, _D]),
    ("nb_set_state", ctypes.c_int, [_H, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D]),
    ("nb_predict", ctypes.c_int, [_H, ctypes.c_double]),
    ("nb_force", ctypes.c_int, [_H, _I, ctypes.c_int, _D, _D, _D]),
    ("nb_force_dev", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    ("nb_force_ext", ctypes.c_int, [_H, ctypes.c_int, _D, _D, _D, _D, _D]),
    ("nb_force_snap", ctypes.c_int, [_H, _I, ctypes.c_int, _D, _D, _D, _D]),
    ("nb_get_snap", ctypes.c_int, [_H, _D, _D]),
    ("nb_set_snap", ctypes.c_int, [_H, _D, _D]),
    ("nb_correct", ctypes.c_int, [_H, _I, ctypes.c_int, ctypes.c_double]),
    ("nb_step", ctypes.c_int, [_H, ctypes.c_double, ctypes.POINTER(nb_stats)]),
    ("nb_energy", ctypes.c_int, [_H, _D, _D]),
    ("nb_get_stats", ctypes.c_int, [_H, ctypes.POINTER(nb_stats)]),
    ("nb_reset_stats", ctypes.c_int, [_H]),
    ("nb_plan_for", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(nb_plan)]),
    ("nb_set_plan_table", ctypes.c_int, [_H, ctypes.POINTER(nb_plan), ctypes.c_int]),
    ("nb_get_plan_table", ctypes.c_int, [_H, ctypes.POINTER(nb_plan)]),
    ("nb_autotune", ctypes.c_int, [_H, ctypes.c_int]),
    ("nb_batch_create", ctypes.c_int, [ctypes.POINTER(nb_config), ctypes.c_int, _I, _D,
                                       ctypes.c_double, ctypes.POINTER(_H)]),
    ("nb_batch_destroy", ctypes.c_int, [_H]),
    ("nb_batch_set", ctypes.c_int, [_H, _D, _D, _D, ctypes.c_double]),
    ("nb_batch_step", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(nb_stats)]),
    ("nb_batch_get", ctypes.c_int, [_H, _D, _D, _D]),
    ("nb_batch_energy", ctypes.c_int, [_H, _D, _D]),
    ("nb_batch_autotune", ctypes.c_int, [_H, _I]),
    ("nb_batch_last_error", ctypes.c_char_p, [_H]),
    ("nb_server_create", ctypes.c_int, [ctypes.POINTER(nb_server_cfg), ctypes.POINTER(_H)]),
    ("nb_server_destroy", ctypes.c_int, [_H]),
    ("nb_submit", ctypes.c_int, [_H, ctypes.POINTER(nb_request), ctypes.POINTER(ctypes.c_uint64)]),
    ("nb_poll", ctypes.c_int, [_H, ctypes.c_uint64, ctypes.POINTER(nb_result)]),
    ("nb_wait", ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(nb_result)]),
    ("nb_cancel", ctypes.c_int, [_H, ctypes.c_uint64]),
    ("nb_result_release", ctypes.c_int, [_H, ctypes.c_uint64]),
    ("nb_server_get_stats", ctypes.c_int, [_H, ctypes.POINTER(nb_server_stats)]),
    ("nb_kick_ext", ctypes.c_int, [_H, _H, ctypes.c_double]),
    ("nb_bridge_step", ctypes.c_int, [_H, _H, ctypes.c_double]),
    ("nb_selftest_wait", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int]),
    ("nb_force_static", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
]


def load(path: str | None = None):
    """Load libnbody.so (raises if it is missing; it is never replaced by a CPU path)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is not built: run `python -m paper_1409_5474_gb300.build`")
            lib = ctypes.CDLL(p)
            for name, res, args in _SIGS:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def declared_symbols():
    """Names of the entry points this binding declares."""
    return [s[0] for s in _SIGS]


def _check(rc, func, h=None):
    if rc != NB_OK:
        lib = load()
        msg = lib.nb_last_error(h)
        raise NBodyError(rc, func, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a, shape):
    out = np.ascontiguousarray(a, dtype=np.float64)
    return out.reshape(shape)


def nb_config_default(**kw) -> nb_config:
    cfg = nb_config()
    load().nb_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        setattr(cfg, k, v)
    return cfg


def nb_version() -> str:
    return load().nb_version().decode()


def nb_status_string(rc: int) -> str:
    return load().nb_status_string(rc).decode()


def nb_create(cfg: nb_config) -> int:
    h = _H()
    rc = load().nb_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(rc, "nb_create", None)
    return h.value


def nb_destroy(h) -> None:
    load().nb_destroy(h)


def nb_set_stream(h, stream_ptr) -> None:
    _check(load().nb_set_stream(h, stream_ptr), "nb_set_stream", h)


def nb_set_particles(h, m, pos, vel, t0=0.0) -> None:
    m = _f64(m, (-1,))
    n = m.shape[0]
    pos = _f64(pos, (3, n))
    vel = _f64(vel, (3, n))
    _check(load().nb_set_particles(h, n, _dp(m), _dp(pos), _dp(vel), float(t0)),
           "nb_set_particles", h)


def nb_init(h) -> None:
    _check(load().nb_init(h), "nb_init", h)


def _n(h) -> int:
    n = ctypes.c_int(0)
    load().nb_get_state(h, ctypes.byref(n), None, None, None, None, None, None, None)
    return n.value


def nb_get_particles(h):
    n = _n(h)
    m = np.empty(n)
    pos = np.empty((3, n))
    vel = np.empty((3, n))
    _check(load().nb_get_particles(h, _dp(m), _dp(pos), _dp(vel)), "nb_get_particles", h)
    return m, pos, vel


def nb_get_state(h):
    """dict with m, pos, vel, acc, jerk (3, n), t, dt (n,)."""
    n = _n(h)
    out = {"m": np.empty(n), "pos": np.empty((3, n)), "vel": np.empty((3, n)),
           "acc": np.empty((3, n)), "jerk": np.empty((3, n)), "t": np.empty(n), "dt": np.empty(n)}
    nn = ctypes.c_int(0)
    _check(load().nb_get_state(h, ctypes.byref(nn), *[_dp(out[k]) for k in
                                                       ("m", "pos", "vel", "acc", "jerk", "t", "dt")]),
           "nb_get_state", h)
    return out


def nb_set_state(h, st) -> None:
    n = np.asarray(st["m"]).shape[0]
    arrs = [_f64(st["m"], (n,)), _f64(st["pos"], (3, n)), _f64(st["vel"], (3, n)),
            _f64(st["acc"], (3, n)), _f64(st["jerk"], (3, n)), _f64(st["t"], (n,)),
            _f64(st["dt"], (n,))]
    _check(load().nb_set_state(h, n, *[_dp(a) for a in arrs]), "nb_set_state", h)


def nb_predict(h, t) -> None:
    _check(load().nb_predict(h, float(t)), "nb_predict", h)


def nb_force(h, idx=None, n_i=None):
    """acc (3, n_i), jerk (3, n_i), pot (n_i,) on members idx (None: all particles)."""
    if idx is None:
        n_i = _n(h) if n_i is None else int(n_i)
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        n_i = idx.shape[0]
        ip = idx.ctypes.data_as(_I)
    acc = np.empty((3, n_i))
    jerk = np.empty((3, n_i))
    pot = np.empty(n_i)
    _check(load().nb_force(h, ip, n_i, _dp(acc), _dp(jerk), _dp(pot)), "nb_force", h)
    return acc, jerk, pot


def nb_force_snap(h, idx=None, n_i=None):
    """Order-6 handles: acc, jerk, snap (3, n_i) and pot (n_i,) on members idx."""
    if idx is None:
        n_i = _n(h) if n_i is None else int(n_i)
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        n_i = idx.shape[0]
        ip = idx.ctypes.data_as(_I)
    acc, jerk, snap = (np.empty((3, n_i)) for _ in range(3))
    pot = np.empty(n_i)
    _check(load().nb_force_snap(h, ip, n_i, _dp(acc), _dp(jerk), _dp(snap), _dp(pot)),
           "nb_force_snap", h)
    return acc, jerk, snap, pot


def nb_get_snap(h):
    """Order-6 handles: (snap, crackle), each (3, n)."""
    n = _n(h)
    snap, crk = np.empty((3, n)), np.empty((3, n))
    _check(load().nb_get_snap(h, _dp(snap), _dp(crk)), "nb_get_snap", h)
    return snap, crk


def nb_set_snap(h, snap, crackle) -> None:
    n = _n(h)
    _check(load().nb_set_snap(h, _dp(_f64(snap, (3, n))), _dp(_f64(crackle, (3, n)))),
           "nb_set_snap", h)


def nb_force_dev(h, idx_ptr, n_i, acc_ptr, jerk_ptr, pot_ptr) -> None:
    """Device-pointer force: pointers are ints (0 for NULL); outputs are (3, n_i) rows."""
    _check(load().nb_force_dev(h, idx_ptr or None, int(n_i), acc_ptr or None, jerk_ptr or None,
                               pot_ptr or None), "nb_force_dev", h)


def nb_force_ext(h, pos, vel):
    pos = _f64(pos, (3, -1))
    n_i = pos.shape[1]
    vel = _f64(vel, (3, n_i))
    acc = np.empty((3, n_i))
    jerk = np.empty((3, n_i))
    pot = np.empty(n_i)
    _check(load().nb_force_ext(h, n_i, _dp(pos), _dp(vel), _dp(acc), _dp(jerk), _dp(pot)),
           "nb_force_ext", h)
    return acc, jerk, pot


def nb_correct(h, idx, t, n_i=None) -> None:
    if idx is None:
        n_i = _n(h) if n_i is None else int(n_i)
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        n_i = idx.shape[0]
        ip = idx.ctypes.data_as(_I)
    _check(load().nb_correct(h, ip, n_i, float(t)), "nb_correct", h)


def nb_step(h, t_end) -> dict:
    st = nb_stats()
    _check(load().nb_step(h, float(t_end), ctypes.byref(st)), "nb_step", h)
    return st.as_dict()


def nb_energy(h):
    k = ctypes.c_double()
    w = ctypes.c_double()
    _check(load().nb_energy(h, ctypes.byref(k), ctypes.byref(w)), "nb_energy", h)
    return k.value, w.value


def nb_get_stats(h) -> dict:
    st = nb_stats()
    _check(load().nb_get_stats(h, ctypes.byref(st)), "nb_get_stats", h)
    return st.as_dict()


def nb_reset_stats(h) -> None:
    _check(load().nb_reset_stats(h), "nb_reset_stats", h)


def nb_plan_for(h, n_i):
    """(kind, nwj, nsplit) of the plan used for n_i i-particles."""
    pl = nb_plan()
    _check(load().nb_plan_for(h, int(n_i), ctypes.byref(pl)), "nb_plan_for", h)
    return pl.as_tuple()


def nb_set_plan_table(h, table):
    """table: list of (kind, nwj, nsplit) per bucket ceil(log2 n_i), or None for the heuristic."""
    if table is None:
        _check(load().nb_set_plan_table(h, None, 0), "nb_set_plan_table", h)
        return
    arr = (nb_plan * len(table))(*[nb_plan(*t) for t in table])
    _check(load().nb_set_plan_table(h, arr, len(table)), "nb_set_plan_table", h)


def nb_get_plan_table(h):
    arr = (nb_plan * 32)()
    _check(load().nb_get_plan_table(h, arr), "nb_get_plan_table", h)
    return [p.as_tuple() for p in arr]


def nb_autotune(h, reps=3):
    _check(load().nb_autotune(h, int(reps)), "nb_autotune", h)
    return nb_get_plan_table(h)


def _bcheck(rc, func, b):
    if rc != NB_OK:
        msg = load().nb_batch_last_error(b) if b else b""
        raise NBodyError(rc, func, (msg or b"").decode() or nb_status_string(rc))


def nb_batch_create(cfg, sizes, eps, dt):
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    b = _H()
    rc = load().nb_batch_create(ctypes.byref(cfg), int(sizes.shape[0]), sizes.ctypes.data_as(_I),
                                _dp(eps), float(dt), ctypes.byref(b))
    if rc != NB_OK:
        raise NBodyError(rc, "nb_batch_create", nb_status_string(rc))
    return b.value


def nb_batch_destroy(b):
    load().nb_batch_destroy(b)


def nb_batch_set(b, m, pos, vel, t0=0.0):
    """m (Ntot,), pos and vel (3, Ntot), concatenated over the systems."""
    m = _f64(m, (-1,))
    n = m.shape[0]
    _bcheck(load().nb_batch_set(b, _dp(m), _dp(_f64(pos, (3, n))), _dp(_f64(vel, (3, n))),
                                float(t0)), "nb_batch_set", b)


def nb_batch_step(b, n_steps):
    st = nb_stats()
    _bcheck(load().nb_batch_step(b, int(n_steps), ctypes.byref(st)), "nb_batch_step", b)
    return st.as_dict()


def nb_batch_get(b, ntot):
    pos = np.empty((3, ntot))
    vel = np.empty((3, ntot))
    t = ctypes.c_double()
    _bcheck(load().nb_batch_get(b, _dp(pos), _dp(vel), ctypes.byref(t)), "nb_batch_get", b)
    return pos, vel, t.value


def nb_batch_energy(b, n_sys):
    k = np.empty(n_sys)
    w = np.empty(n_sys)
    _bcheck(load().nb_batch_energy(b, _dp(k), _dp(w)), "nb_batch_energy", b)
    return k, w


def nb_batch_autotune(b):
    t = ctypes.c_int()
    _bcheck(load().nb_batch_autotune(b, ctypes.byref(t)), "nb_batch_autotune", b)
    return t.value


def nb_selftest_wait(which, limit_s, device=0) -> int:
    """Run one bounded device wait that nothing completes; returns the status
    (NB_ERR_TIMEOUT is the expected one)."""
    return load().nb_selftest_wait(int(which), float(limit_s), int(device))


def nb_kick_ext(target, field, dt_kick) -> None:
    _check(load().nb_kick_ext(target, field, float(dt_kick)), "nb_kick_ext", target)


def nb_bridge_step(a, b, dt) -> None:
    _check(load().nb_bridge_step(a, b, float(dt)), "nb_bridge_step", a)


class Batch:
    """Many independent systems advanced with shared-step Hermite on the GPU."""

    def __init__(self, systems, eps, dt, **cfg):
        """systems: list of ic.Particles (or objects with m, pos (n,3), vel (n,3))."""
        self.sizes = np.array([len(p.m) for p in systems], dtype=np.int32)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.ntot = int(self.sizes.sum())
        self.cfg = nb_config_default(**cfg)
        self.b = nb_batch_create(self.cfg, self.sizes, eps, dt)
        try:
            m = np.concatenate([np.asarray(p.m, dtype=np.float64) for p in systems])
            pos = np.concatenate([np.asarray(p.pos, dtype=np.float64) for p in systems]).T
            vel = np.concatenate([np.asarray(p.vel, dtype=np.float64) for p in systems]).T
            nb_batch_set(self.b, m, pos, vel)
        except Exception:
            self.close()
            raise

    def close(self):
        if getattr(self, "b", None):
            nb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n_steps):
        return nb_batch_step(self.b, n_steps)

    def get(self):
        return nb_batch_get(self.b, self.ntot)

    def system(self, s, arr):
        """Columns of system s in a (3, Ntot) array."""
        o = self.offsets[s]
        return arr[:, o:o + self.sizes[s]]

    def energy(self):
        return nb_batch_energy(self.b, len(self.sizes))

    def autotune(self):
        return nb_batch_autotune(self.b)


def _scheck(rc, func):
    if rc != NB_OK:
        raise NBodyError(rc, func, nb_status_string(rc))


def nb_server_create(device=0, variant=NB_F32DS, budget_bytes=0, max_inflight=0, max_queue=0,
                     eta=0.0, dt_max=0.0, flags=0):
    cfg = nb_server_cfg(int(device), int(variant), int(budget_bytes), int(max_inflight),
                        int(max_queue), float(eta), float(dt_max), int(flags))
    srv = _H()
    _scheck(load().nb_server_create(ctypes.byref(cfg), ctypes.byref(srv)), "nb_server_create")
    return srv.value


def nb_server_destroy(srv) -> None:
    load().nb_server_destroy(srv)


def nb_submit(srv, kind, m, pos, vel, eps, t_span=0.0) -> int:
    """Queue a request; m (n,), pos and vel (3, n). Returns the ticket."""
    m = _f64(m, (-1,))
    n = m.shape[0]
    pos = _f64(pos, (3, n))
    vel = _f64(vel, (3, n))
    req = nb_request(int(kind), n, _dp(m), _dp(pos), _dp(vel), float(eps), float(t_span))
    t = ctypes.c_uint64()
    _scheck(load().nb_submit(srv, ctypes.byref(req), ctypes.byref(t)), "nb_submit")
    return t.value


def _result_dict(r: nb_result) -> dict:
    d = {k: getattr(r, k) for k in ("status", "error", "n", "t_submit", "t_start", "t_done",
                                     "interactions", "block_steps")}
    n = r.n
    for k, rows in (("acc", 3), ("jerk", 3), ("pot", 1), ("pos", 3), ("vel", 3)):
        p = getattr(r, k)
        if p:
            a = np.ctypeslib.as_array(p, shape=(rows * n,)).copy()
            d[k] = a.reshape(3, n) if rows == 3 else a
    return d


def nb_poll(srv, ticket) -> dict:
    r = nb_result()
    _scheck(load().nb_poll(srv, int(ticket), ctypes.byref(r)), "nb_poll")
    return _result_dict(r)


def nb_wait(srv, ticket, timeout_s=60.0) -> dict:
    """Wait for a request; raises NBodyError(NB_ERR_TIMEOUT) if it is not done in time."""
    r = nb_result()
    _scheck(load().nb_wait(srv, int(ticket), float(timeout_s), ctypes.byref(r)), "nb_wait")
    return _result_dict(r)


def nb_cancel(srv, ticket) -> None:
    _scheck(load().nb_cancel(srv, int(ticket)), "nb_cancel")


def nb_result_release(srv, ticket) -> None:
    _scheck(load().nb_result_release(srv, int(ticket)), "nb_result_release")


def nb_server_get_stats(srv) -> dict:
    st = nb_server_stats()
    _scheck(load().nb_server_get_stats(srv, ctypes.byref(st)), "nb_server_get_stats")
    return st.as_dict()


class Server:
    """Continuous-batching force / integration service on one GPU."""

    def __init__(self, **cfg):
        self.s = nb_server_create(**cfg)

    def close(self):
        if getattr(self, "s", None):
            nb_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def force(self, m, pos, vel, eps) -> int:
        return nb_submit(self.s, NB_REQ_FORCE, m, pos, vel, eps)

    def evolve(self, m, pos, vel, eps, t_span) -> int:
        return nb_submit(self.s, NB_REQ_EVOLVE, m, pos, vel, eps, t_span)

    def poll(self, ticket) -> dict:
        return nb_poll(self.s, ticket)

    def wait(self, ticket, timeout_s=60.0, release=True) -> dict:
        d = nb_wait(self.s, ticket, timeout_s)
        if release:
            nb_result_release(self.s, ticket)
        return d

    def cancel(self, ticket) -> None:
        nb_cancel(self.s, ticket)

    def release(self, ticket) -> None:
        nb_result_release(self.s, ticket)

    def stats(self) -> dict:
        return nb_server_get_stats(self.s)


NB_STATIC_MAX_NI = 1024


def nb_force_static(n_j, m_ptr, pos_ptr, vel_ptr, ld, n_i, idx_ptr, eps, acc_ptr, jerk_ptr,
                    pot_ptr, stream_ptr=0) -> None:
    """Allocation-free FP64 force on caller-owned device buffers (pointers as ints, 0 = NULL).
    For callers that cannot allocate device memory; see nbody.h."""
    rc = load().nb_force_static(int(n_j), m_ptr, pos_ptr, vel_ptr, int(ld), int(n_i),
                                idx_ptr or None, float(eps), acc_ptr or None, jerk_ptr or None,
                                pot_ptr or None, stream_ptr or None)
    if rc != NB_OK:
        raise NBodyError(rc, "nb_force_static", nb_status_string(rc))


class System:
    """One N-body system on the GPU (owns an nb_handle)."""

    def __init__(self, m, pos, vel, t0=0.0, n_max=None, **cfg):
        """m (n,), pos and vel (n, 3) as ``ic.Particles`` holds them; cfg: nb_config fields."""
        m = np.asarray(m, dtype=np.float64)
        n = m.shape[0]
        cfg.setdefault("n_max", n if n_max is None else n_max)
        self.cfg = nb_config_default(**cfg)
        self.h = nb_create(self.cfg)
        try:
            nb_set_particles(self.h, m, _f64(pos, (n, 3)).T, _f64(vel, (n, 3)).T, t0)
        except Exception:
            self.close()
            raise

    def close(self):
        if getattr(self, "h", None):
            nb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def predict(self, t):
        nb_predict(self.h, t)

    def force(self, idx=None):
        return nb_force(self.h, idx)

    def force_ext(self, pos, vel):
        return nb_force_ext(self.h, pos, vel)

    def force_snap(self, idx=None):
        return nb_force_snap(self.h, idx)

    def snap(self):
        return nb_get_snap(self.h)

    def set_snap(self, snap, crackle):
        nb_set_snap(self.h, snap, crackle)

    def correct(self, idx, t):
        nb_correct(self.h, idx, t)

    def step(self, t_end):
        return nb_step(self.h, t_end)

    def energy(self):
        return nb_energy(self.h)

    def state(self):
        return nb_get_state(self.h)

    def set_state(self, st):
        nb_set_state(self.h, st)
