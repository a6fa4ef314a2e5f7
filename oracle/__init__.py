"""FP64 CPU oracle for the direct-summation Hermite hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never loads it and
has no CPU fallback; the two share no code. The arithmetic lives in
``oracle.c`` (plain C, binary64); this module compiles it with gcc on first use
and marshals numpy arrays through ctypes.

Every routine follows a passage of the paper (Portegies Zwart & Bedorf,
"Computational Gravitational Dynamics with Modern Numerical Accelerators"):

- ``force`` / ``force_ext``: direct summation of softened gravity from the
  j-set onto an i-set that is part of it or disjoint from it (Sect. III.A);
- ``predict``: prediction of the j particles to the block time (Sect. III.A);
- ``correct_one``, ``aarseth_dt``, ``initial_dt``, ``quantize``: the
  4th-order Hermite predictor-corrector with individual block steps
  (Sect. II, III, VI);
- ``hermite_run``: the block-step (or shared-step) integration loop;
- ``force6``, ``predict6``, ``correct6_one``, ``aarseth6_dt``, ``hermite6_run``: the
  6th-order Hermite scheme (acc, jerk and snap per pair; Sect. II, the >= 4th-order
  integrators with individual steps that direct codes use);
- ``kick``, ``bridge_run``: the 2nd-order kick-drift-kick coupling of two
  systems (Sect. V, the Hamiltonian split behind the hybrid codes), composed
  of ``force_ext``, ``force`` and ``hermite_run``;
- ``energy``: kinetic plus softened potential energy.

Parity pins live in ``tests/test_oracle_*.py``; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


# gcc flags of the oracle: binary64 as written (no FMA contraction, no fast-math, no
# reassociation), so the x86 build host and the Arm GPU host compute the same bits; no
# -march=native for the same reason.
CFLAGS = "-O3 -std=c11 -fopenmp -ffp-contract=off -fno-fast-math"


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source with CFLAGS into a shared library."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = (["gcc"] + CFLAGS.split() + ["-fPIC", "-shared", "-Wall", "-o", tmp, src, "-lm"])
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def use_library(path=None):
    """Point the wrapper at another build of oracle.c (a planted-mistake copy in the
    mutation tests); None restores the default library. Returns the previous one."""
    global _lib
    with _lock:
        prev = _lib
        _lib = None if path is None else _bind(ctypes.CDLL(path))
    return prev


def _restore(lib):
    global _lib
    with _lock:
        _lib = lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.orc_force_idx.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                  _I, _D, _D, _D]
    lib.orc_force_ext.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, ctypes.c_int,
                                  _D, _D, _D, _D, _D]
    lib.orc_predict.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, _D, _D, _D, _D, _D]
    lib.orc_correct_one.argtypes = [ctypes.c_double] + [_D] * 10
    lib.orc_aarseth_dt.argtypes = [_D, _D, _D, _D, ctypes.c_double]
    lib.orc_aarseth_dt.restype = ctypes.c_double
    lib.orc_initial_dt.argtypes = [_D, _D, ctypes.c_double]
    lib.orc_initial_dt.restype = ctypes.c_double
    lib.orc_quantize.argtypes = [ctypes.c_double] * 5
    lib.orc_quantize.restype = ctypes.c_double
    lib.orc_hermite_run.argtypes = ([ctypes.c_int, _D, _D, _D, _D, _D, _D, _D]
                                    + [ctypes.c_double] * 7
                                    + [ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_long), _D])
    lib.orc_hermite_run.restype = ctypes.c_int
    lib.orc_energy.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, _D, _D]
    lib.orc_force6_idx.argtypes = [ctypes.c_int, _D, _D, _D, _D, ctypes.c_double,
                                   ctypes.c_int, _I, _D, _D, _D, _D]
    lib.orc_predict6.argtypes = [ctypes.c_int, ctypes.c_double] + [_D] * 10
    lib.orc_correct6_one.argtypes = [ctypes.c_double] + [_D] * 13
    lib.orc_hermite6_run.argtypes = ([ctypes.c_int] + [_D] * 9
                                     + [ctypes.c_double] * 7
                                     + [ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong,
                                        ctypes.c_double]
                                     + [ctypes.c_long, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_long), _D])
    lib.orc_aarseth6_dt.argtypes = [_D] * 6 + [ctypes.c_double]
    lib.orc_aarseth6_dt.restype = ctypes.c_double
    lib.orc_hermite6_run.restype = ctypes.c_int
    lib.orc_num_threads.restype = ctypes.c_int
    return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(_D)


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS, else all cores)."""
    return int(_load().orc_num_threads())


def force(m, pos, vel, eps2, idx=None):
    """acc, jerk (ni,3) and pot (ni,) on i = idx[k] (all if None) from every j != i."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    pos = _f64(pos, (n, 3))
    vel = _f64(vel, (n, 3))
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.size and (idx.min() < 0 or idx.max() >= n):
            raise IndexError("idx out of range")
        ni, ip = idx.shape[0], idx.ctypes.data_as(_I)
    acc = np.zeros((ni, 3))
    jerk = np.zeros((ni, 3))
    pot = np.zeros(ni)
    lib.orc_force_idx(n, _p(m), _p(pos), _p(vel), float(eps2), ni, ip, _p(acc), _p(jerk), _p(pot))
    return acc, jerk, pot


def force_ext(m, pos, vel, eps2, ipos, ivel):
    """acc, jerk, pot on an external i-set (no self-exclusion)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    pos = _f64(pos, (n, 3))
    vel = _f64(vel, (n, 3))
    ipos = _f64(ipos).reshape(-1, 3)
    ivel = _f64(ivel, ipos.shape)
    ni = ipos.shape[0]
    acc = np.zeros((ni, 3))
    jerk = np.zeros((ni, 3))
    pot = np.zeros(ni)
    lib.orc_force_ext(n, _p(m), _p(pos), _p(vel), float(eps2), ni, _p(ipos), _p(ivel),
                      _p(acc), _p(jerk), _p(pot))
    return acc, jerk, pot


def predict(t, tj, pos, vel, acc, jerk):
    """Predicted (pos, vel) of every particle at time t from its own time tj."""
    lib = _load()
    tj = _f64(tj)
    n = tj.shape[0]
    pos, vel, acc, jerk = (_f64(a, (n, 3)) for a in (pos, vel, acc, jerk))
    pp = np.zeros((n, 3))
    vp = np.zeros((n, 3))
    lib.orc_predict(n, float(t), _p(tj), _p(pos), _p(vel), _p(acc), _p(jerk), _p(pp), _p(vp))
    return pp, vp


def correct_one(dt, xp, vp, a0, j0, a1, j1):
    """Hermite corrector for one particle: (x1, v1, a2_end, a3_end)."""
    lib = _load()
    args = [_f64(a, (3,)) for a in (xp, vp, a0, j0, a1, j1)]
    outs = [np.zeros(3) for _ in range(4)]
    lib.orc_correct_one(float(dt), *[_p(a) for a in args], *[_p(o) for o in outs])
    return tuple(outs)


def aarseth_dt(a, j, a2, a3, eta):
    lib = _load()
    return float(lib.orc_aarseth_dt(*[_p(_f64(v, (3,))) for v in (a, j, a2, a3)], float(eta)))


def initial_dt(a, j, eta_s):
    lib = _load()
    return float(lib.orc_initial_dt(_p(_f64(a, (3,))), _p(_f64(j, (3,))), float(eta_s)))


def quantize(dt_raw, dt_old, t_new, dt_min, dt_max):
    return float(_load().orc_quantize(float(dt_raw), float(dt_old), float(t_new), float(dt_min),
                                      float(dt_max)))


class State:
    """Integrator state of one system (copies of the caller's arrays)."""

    def __init__(self, m, pos, vel, t0=0.0, acc=None, jerk=None, t=None, dt=None):
        self.m = _f64(m).copy()
        n = self.m.shape[0]
        self.pos = _f64(pos, (n, 3)).copy()
        self.vel = _f64(vel, (n, 3)).copy()
        self.acc = np.zeros((n, 3)) if acc is None else _f64(acc, (n, 3)).copy()
        self.jerk = np.zeros((n, 3)) if jerk is None else _f64(jerk, (n, 3)).copy()
        self.t = np.full(n, float(t0)) if t is None else _f64(t).copy()
        self.dt = np.zeros(n) if dt is None else _f64(dt).copy()
        self.initialised = acc is not None

    @property
    def n(self):
        return self.m.shape[0]


def hermite_run(state: State, t_end, eps2, eta=0.01, eta_s=None, dt_min=2.0 ** -30,
                dt_max=1.0 / 16, dt_shared=0.0, max_steps=0, n_corr=1):
    """Advance ``state`` in place with block (or shared, dt_shared > 0) steps to t_end;
    n_corr force evaluations and corrections per step (1: PEC, 2: P(EC)^2, ...).

    Returns (n_block_steps, n_interactions)."""
    lib = _load()
    if eta_s is None:
        eta_s = eta
    steps = ctypes.c_long(0)
    inter = ctypes.c_double(0.0)
    init = 0 if state.initialised else 1
    rc = lib.orc_hermite_run(state.n, _p(state.m), _p(state.pos), _p(state.vel), _p(state.acc),
                             _p(state.jerk), _p(state.t), _p(state.dt), float(eps2), float(eta),
                             float(eta_s), float(dt_min), float(dt_max), float(dt_shared),
                             float(t_end), int(max_steps), init, int(n_corr),
                             ctypes.byref(steps), ctypes.byref(inter))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    state.initialised = True
    return int(steps.value), float(inter.value)


def kick(state: State, field: State, eps2_field, eps2_self, dt_kick):
    """Bridge kick (Sect. V): the velocities of ``state`` (synchronised) change by dt_kick
    times the acceleration of the ``field`` system at their positions (softening of the
    field), then acc and jerk of ``state``'s own particles are evaluated again at the new
    velocities; the particles' steps are kept."""
    acc, _, _ = force_ext(field.m, field.pos, field.vel, eps2_field, state.pos, state.vel)
    state.vel += dt_kick * acc
    a, j, _ = force(state.m, state.pos, state.vel, eps2_self)
    state.acc[:] = a
    state.jerk[:] = j


def bridge_run(sa: State, sb: State, eps2_a, eps2_b, dt, n_steps, **hermite_kw):
    """n_steps kick-drift-kick bridge steps of two systems (Sect. V, 2nd order): each
    system is kicked by the other's field for dt/2, evolves with its own Hermite
    integrator (``hermite_run`` keywords) for dt, and is kicked again. Both systems start
    synchronised at the same time; uninitialised ones are initialised first."""
    for st, e2 in ((sa, eps2_a), (sb, eps2_b)):
        if not st.initialised:
            hermite_run(st, float(st.t[0]), e2, **hermite_kw)
    for _ in range(n_steps):
        t = float(sa.t[0])
        kick(sa, sb, eps2_b, eps2_a, 0.5 * dt)
        kick(sb, sa, eps2_a, eps2_b, 0.5 * dt)
        hermite_run(sa, t + dt, eps2_a, **hermite_kw)
        hermite_run(sb, t + dt, eps2_b, **hermite_kw)
        kick(sa, sb, eps2_b, eps2_a, 0.5 * dt)
        kick(sb, sa, eps2_a, eps2_b, 0.5 * dt)


def force6(m, pos, vel, acc_j, eps2, idx=None):
    """acc, jerk, snap (ni,3) and pot (ni,) on i = idx[k] (all if None) from every j != i,
    with acc_j (n,3) the particles' accelerations (the snap differentiates along them)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    pos, vel, acc_j = (_f64(a, (n, 3)) for a in (pos, vel, acc_j))
    if idx is None:
        ni, ip = n, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.size and (idx.min() < 0 or idx.max() >= n):
            raise IndexError("idx out of range")
        ni, ip = idx.shape[0], idx.ctypes.data_as(_I)
    acc, jerk, snap = (np.zeros((ni, 3)) for _ in range(3))
    pot = np.zeros(ni)
    lib.orc_force6_idx(n, _p(m), _p(pos), _p(vel), _p(acc_j), float(eps2), ni, ip, _p(acc),
                       _p(jerk), _p(snap), _p(pot))
    return acc, jerk, snap, pot


def predict6(t, tj, pos, vel, acc, jerk, snap, crackle):
    """Predicted (pos, vel, acc) at time t through the crackle term."""
    lib = _load()
    tj = _f64(tj)
    n = tj.shape[0]
    ins = [_f64(a, (n, 3)) for a in (pos, vel, acc, jerk, snap, crackle)]
    outs = [np.zeros((n, 3)) for _ in range(3)]
    lib.orc_predict6(n, float(t), _p(tj), *[_p(a) for a in ins], *[_p(o) for o in outs])
    return tuple(outs)


def correct6_one(dt, x0, v0, a0, j0, s0, a1, j1, s1):
    """6th-order Hermite corrector for one particle: (x1, v1, a3_end, a4_end, a5_end)."""
    lib = _load()
    args = [_f64(a, (3,)) for a in (x0, v0, a0, j0, s0, a1, j1, s1)]
    outs = [np.zeros(3) for _ in range(5)]
    lib.orc_correct6_one(float(dt), *[_p(a) for a in args], *[_p(o) for o in outs])
    return tuple(outs)


class State6(State):
    """State of the 6th-order scheme: State plus snap and crackle per particle."""

    def __init__(self, m, pos, vel, t0=0.0, acc=None, jerk=None, snap=None, crackle=None,
                 t=None, dt=None):
        super().__init__(m, pos, vel, t0, acc, jerk, t, dt)
        n = self.n
        self.snap = np.zeros((n, 3)) if snap is None else _f64(snap, (n, 3)).copy()
        self.crackle = np.zeros((n, 3)) if crackle is None else _f64(crackle, (n, 3)).copy()


CRITERIA6 = {"aarseth": 0, "generalised": 1}


def aarseth6_dt(a, a1, a2, a3, a4, a5, eta):
    """The published order-6 step criterion (Aarseth's form generalised to a .. a5)."""
    lib = _load()
    return float(lib.orc_aarseth6_dt(*[_p(_f64(v, (3,))) for v in (a, a1, a2, a3, a4, a5)],
                                     float(eta)))


def hermite6_run(state: State6, t_end, eps2, eta=0.02, eta_s=0.01, dt_min=2.0 ** -30,
                 dt_max=1.0 / 16, dt_shared=0.0, max_steps=0, noise=0.0, criterion="aarseth",
                 perturb=0.0, seed=0):
    """Advance ``state`` in place with the 6th-order Hermite scheme and block (or shared)
    steps to t_end; ``noise``: the forces' relative rounding noise, which sets the floor
    under the crackle in the step criterion (0: exact forces, no floor).
    ``criterion``: "aarseth" (Aarseth's form on a, jerk, snap, crackle; the default) or
    "generalised" (the published order-6 criterion on a .. a5; ``noise`` unused).
    ``perturb`` > 0: seeded relative noise of that size on every evaluated a, jerk and snap
    of the block steps (a model of reduced-precision forces for the criterion study).
    Returns (n_block_steps, n_interactions)."""
    lib = _load()
    steps = ctypes.c_long(0)
    inter = ctypes.c_double(0.0)
    init = 0 if state.initialised else 1
    rc = lib.orc_hermite6_run(state.n, _p(state.m), _p(state.pos), _p(state.vel),
                              _p(state.acc), _p(state.jerk), _p(state.snap),
                              _p(state.crackle), _p(state.t), _p(state.dt), float(eps2),
                              float(eta), float(eta_s), float(dt_min), float(dt_max),
                              float(dt_shared), float(noise), CRITERIA6[criterion],
                              float(perturb), int(seed), float(t_end), int(max_steps), init,
                              ctypes.byref(steps), ctypes.byref(inter))
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    state.initialised = True
    return int(steps.value), float(inter.value)


def energy(m, pos, vel, eps2):
    """(K, W): kinetic and softened potential energy (pairwise sum over i<j)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    kin = ctypes.c_double()
    w = ctypes.c_double()
    lib.orc_energy(n, _p(m), _p(_f64(pos, (n, 3))), _p(_f64(vel, (n, 3))), float(eps2),
                   ctypes.byref(kin), ctypes.byref(w))
    return float(kin.value), float(w.value)
