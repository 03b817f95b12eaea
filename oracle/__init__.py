"""FP64 CPU oracle of the Hermite-4 (and Hermite-6) block-step integrators -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library behind ``include/gravidy.h`` and its Python binding) never calls it.

The arithmetic lives in ``hermite_oracle.c`` and ``hermite6_oracle.c`` (plain
single-threaded C, compiled without FMA contraction); this module compiles them
on first use with gcc and wraps them with ctypes.  Every function cites the part of GraviDy
(arXiv 1702.00440) it follows in the C source.

Conventions: positions/velocities/accelerations/jerks are ``float64`` arrays of
shape ``(n, 3)``; times are integer ticks of ``dt_min``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "hermite_oracle.c"), os.path.join(_HERE, "hermite6_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle sources into ``_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(q) for q in _SRCS):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_force": (None, [_I64, _P, _P, _P, _D, _I64, _P, _P, _P]),
            "or_force_absnorm": (None, [_I64, _P, _P, _P, _D, _I64, _P, _P, _P]),
            "or_energy": (None, [_I64, _P, _P, _P, _D, _P, _P]),
            "or_active": (_I64, [_I64, _P, _P, _P]),
            "or_predict_one": (None, [_P, _P, _P, _P, _D, _P, _P]),
            "or_predict_all": (None, [_I64, _P, _P, _P, _P, _P, _P, _P]),
            "or_hermite_derivs": (None, [_P, _P, _P, _P, _D, _P, _P]),
            "or_correct_one": (None, [_P, _P, _P, _P, _D, _P, _P]),
            "or_aarseth_dt": (_D, [_P, _P, _P, _P, _D]),
            "or_quantise_init": (_I64, [_D, _D, _I64]),
            "or_quantise": (_I64, [_D, _I64, _I64, _D, _I64]),
            "or_sim_new": (_P, [_I64, _P, _P, _P, _D, _D, _D, _D, _I64]),
            "or_sim_free": (None, [_P]),
            "or_sim_step": (_I64, [_P, _P, _P]),
            "or_sim_replay": (None, [_P, _I64, _I64, _P]),
            "or_sim_evolve": (_I64, [_P, _I64]),
            "or_sim_energy": (None, [_P, _P, _P]),
            "or_sim_get": (None, [_P, _P, _P, _P, _P, _P, _P]),
            "or_sim_stats": (None, [_P, _P, _P, _P, _P]),
            "or_pn_accel": (None, [_D, _D, _P, _P, _D, ctypes.c_int, _P]),
            "or_pn_jerk": (None, [_D, _D, _P, _P, _P, _D, ctypes.c_int, _P]),
            "or_sim_set_pn": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D, ctypes.c_int]),
            "or6_force": (None, [_I64, _P, _P, _P, _P, _D, _I64, _P, _P, _P, _P]),
            "or6_predict_one": (None, [_P, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
            "or6_correct_one": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _D, _P, _P]),
            "or6_derivs": (None, [_P, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
            "or6_aarseth_dt": (_D, [_P, _P, _P, _P, _P, _P, _D]),
            "or4s_correct_one": (None, [_P, _P, _P, _P, _P, _P, _D, _P, _P]),
            "or6_sim_new": (_P, [_I64, _P, _P, _P, _D, _D, _D, _D, _D, _I64, ctypes.c_int, ctypes.c_int]),
            "or6_sim_free": (None, [_P]),
            "or6_sim_step": (_I64, [_P, _P, _P]),
            "or6_sim_replay": (None, [_P, _I64, _I64, _P]),
            "or6_sim_evolve": (_I64, [_P, _I64]),
            "or6_sim_energy": (None, [_P, _P, _P]),
            "or6_sim_get": (None, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
            "or6_sim_stats": (None, [_P, _P, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def force(m, x, v, eps, idx=None):
    """Softened acceleration and jerk of particles ``idx`` (default: all)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, np.int32)
    k = idx.shape[0]
    acc = np.zeros((k, 3))
    jrk = np.zeros((k, 3))
    lib.or_force(n, _ptr(m), _ptr(x), _ptr(v), float(eps) ** 2, k, _ptr(idx), _ptr(acc), _ptr(jrk))
    return acc, jrk


def force_absnorm(m, x, v, eps, idx=None):
    """Per-particle sums of term magnitudes (tolerance scales)."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, np.int32)
    k = idx.shape[0]
    an = np.zeros(k)
    jn = np.zeros(k)
    lib.or_force_absnorm(n, _ptr(m), _ptr(x), _ptr(v), float(eps) ** 2, k, _ptr(idx), _ptr(an), _ptr(jn))
    return an, jn


def energy(m, x, v, eps):
    """(K, U) with the softened potential."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    K = ctypes.c_double()
    U = ctypes.c_double()
    lib.or_energy(n, _ptr(m), _ptr(x), _ptr(v), float(eps) ** 2, ctypes.byref(K), ctypes.byref(U))
    return K.value, U.value


def active(tnext):
    """(ascending active indices, t_next) for an int64 next-time array."""
    lib = _load()
    t = np.ascontiguousarray(tnext, dtype=np.int64)
    idx = np.zeros(t.shape[0], np.int32)
    tn = ctypes.c_int64()
    c = lib.or_active(t.shape[0], _ptr(t), _ptr(idx), ctypes.byref(tn))
    return idx[:c].copy(), tn.value


def predict_one(x, v, a, j, dt):
    lib = _load()
    xp = np.zeros(3)
    vp = np.zeros(3)
    lib.or_predict_one(_ptr(_f64(x)), _ptr(_f64(v)), _ptr(_f64(a)), _ptr(_f64(j)), float(dt), _ptr(xp), _ptr(vp))
    return xp, vp


def predict_all(x, v, a, j, dt):
    """Taylor prediction of every particle i over dt[i]."""
    lib = _load()
    dt = _f64(dt)
    n = dt.shape[0]
    x, v, a, j = (_f64(q, (n, 3)) for q in (x, v, a, j))
    xp = np.zeros((n, 3))
    vp = np.zeros((n, 3))
    lib.or_predict_all(n, _ptr(x), _ptr(v), _ptr(a), _ptr(j), _ptr(dt), _ptr(xp), _ptr(vp))
    return xp, vp


def hermite_derivs(a0, j0, a1, j1, dt):
    lib = _load()
    a2 = np.zeros(3)
    a3 = np.zeros(3)
    lib.or_hermite_derivs(_ptr(_f64(a0)), _ptr(_f64(j0)), _ptr(_f64(a1)), _ptr(_f64(j1)), float(dt), _ptr(a2), _ptr(a3))
    return a2, a3


def correct_one(xp, vp, a2, a3, dt):
    lib = _load()
    x1 = np.zeros(3)
    v1 = np.zeros(3)
    lib.or_correct_one(_ptr(_f64(xp)), _ptr(_f64(vp)), _ptr(_f64(a2)), _ptr(_f64(a3)), float(dt), _ptr(x1), _ptr(v1))
    return x1, v1


def aarseth_dt(a1, j1, a2e, a3e, eta):
    lib = _load()
    return lib.or_aarseth_dt(_ptr(_f64(a1)), _ptr(_f64(j1)), _ptr(_f64(a2e)), _ptr(_f64(a3e)), float(eta))


def quantise_init(dt, dt_min, dtau_max):
    return _load().or_quantise_init(float(dt), float(dt_min), int(dtau_max))


def quantise(dt_new, dtau_old, tick_now, dt_min, dtau_max):
    return _load().or_quantise(float(dt_new), int(dtau_old), int(tick_now), float(dt_min), int(dtau_max))


PN_1 = 1     # 1PN terms of the pair
PN_2 = 2     # 2PN terms of the pair
PN_25 = 4    # 2.5PN (radiation reaction) terms of the pair


def pn_accel(mp, mq, r, v, c, terms=PN_1 | PN_2 | PN_25):
    """Post-Newtonian relative acceleration of a pair (r = x_p - x_q, v = v_p - v_q)."""
    a = np.zeros(3)
    _load().or_pn_accel(float(mp), float(mq), _ptr(_f64(r)), _ptr(_f64(v)), float(c), int(terms), _ptr(a))
    return a


def pn_jerk(mp, mq, r, v, arel, c, terms=PN_1 | PN_2 | PN_25):
    """Time derivative of pn_accel along the relative motion (dv/dt = arel)."""
    j = np.zeros(3)
    _load().or_pn_jerk(float(mp), float(mq), _ptr(_f64(r)), _ptr(_f64(v)), _ptr(_f64(arel)), float(c), int(terms),
                       _ptr(j))
    return j


class Sim:
    """The oracle integrator (GraviDy Sec. 2.4 steps 1-7)."""

    def __init__(self, m, x, v, eps, eta, dt_min=2.0 ** -22, dt_max=0.125, fixed_dtau=0):
        self._lib = _load()
        m = _f64(m)
        self.n = n = m.shape[0]
        self.dt_min = float(dt_min)
        self.dt_max = float(dt_max)
        x = _f64(x, (n, 3))
        v = _f64(v, (n, 3))
        h = self._lib.or_sim_new(n, _ptr(m), _ptr(x), _ptr(v), float(eps), float(eta), self.dt_min, self.dt_max, int(fixed_dtau))
        if not h:
            raise ValueError("oracle rejected the arguments")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_sim_free(h)
            self._h = None

    def set_pn(self, p, q, c, terms=PN_1 | PN_2 | PN_25):
        """Post-Newtonian terms for the pair (p, q), before the first step."""
        if self._lib.or_sim_set_pn(self._h, int(p), int(q), float(c), int(terms)) != 0:
            raise ValueError("oracle rejected the post-Newtonian pair")

    def step(self):
        """One free-running block step -> (tick, ascending active indices)."""
        idx = np.zeros(self.n, np.int32)
        t = ctypes.c_int64()
        c = self._lib.or_sim_step(self._h, ctypes.byref(t), _ptr(idx))
        return t.value, idx[:c].copy()

    def replay(self, tick, idx):
        idx = np.ascontiguousarray(idx, np.int32)
        self._lib.or_sim_replay(self._h, int(tick), idx.shape[0], _ptr(idx))

    def evolve_ticks(self, tick_end):
        return self._lib.or_sim_evolve(self._h, int(tick_end))

    def evolve(self, t_end):
        return self.evolve_ticks(int(round(t_end / self.dt_min)))

    def energy(self):
        K = ctypes.c_double()
        U = ctypes.c_double()
        self._lib.or_sim_energy(self._h, ctypes.byref(K), ctypes.byref(U))
        return K.value, U.value

    def state(self):
        n = self.n
        x, v, a, j = (np.zeros((n, 3)) for _ in range(4))
        tau = np.zeros(n, np.int64)
        dtau = np.zeros(n, np.int64)
        self._lib.or_sim_get(self._h, _ptr(x), _ptr(v), _ptr(a), _ptr(j), _ptr(tau), _ptr(dtau))
        return dict(x=x, v=v, a=a, j=j, tau=tau, dtau=dtau)

    def stats(self):
        t = ctypes.c_int64()
        nb = ctypes.c_int64()
        ns = ctypes.c_int64()
        it = ctypes.c_double()
        self._lib.or_sim_stats(self._h, ctypes.byref(t), ctypes.byref(nb), ctypes.byref(ns), ctypes.byref(it))
        return dict(tick=t.value, nblock=nb.value, nsteps=ns.value, interactions=it.value)


# ---------------------------------------------------------------- sixth order

def force6(m, x, v, a, eps, idx=None):
    """Softened acceleration, jerk and snap of particles ``idx`` (default: all)
    from positions, velocities and accelerations of all particles."""
    lib = _load()
    m = _f64(m)
    n = m.shape[0]
    x, v, a = (_f64(q, (n, 3)) for q in (x, v, a))
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, np.int32)
    k = idx.shape[0]
    acc, jrk, snp = np.zeros((k, 3)), np.zeros((k, 3)), np.zeros((k, 3))
    lib.or6_force(n, _ptr(m), _ptr(x), _ptr(v), _ptr(a), float(eps) ** 2, k, _ptr(idx), _ptr(acc), _ptr(jrk),
                  _ptr(snp))
    return acc, jrk, snp


def predict6_one(x, v, a, j, s, c, dt):
    lib = _load()
    xp, vp, ap = np.zeros(3), np.zeros(3), np.zeros(3)
    lib.or6_predict_one(*(_ptr(_f64(q)) for q in (x, v, a, j, s, c)), float(dt), _ptr(xp), _ptr(vp), _ptr(ap))
    return xp, vp, ap


def correct6_one(x0, v0, a0, j0, s0, a1, j1, s1, dt):
    lib = _load()
    x1, v1 = np.zeros(3), np.zeros(3)
    lib.or6_correct_one(*(_ptr(_f64(q)) for q in (x0, v0, a0, j0, s0, a1, j1, s1)), float(dt), _ptr(x1), _ptr(v1))
    return x1, v1


def correct4s_one(x0, v0, a0, j0, a1, j1, dt):
    """Time-symmetric fourth-order corrector (Hut, Makino & McMillan 1995)."""
    lib = _load()
    x1, v1 = np.zeros(3), np.zeros(3)
    lib.or4s_correct_one(*(_ptr(_f64(q)) for q in (x0, v0, a0, j0, a1, j1)), float(dt), _ptr(x1), _ptr(v1))
    return x1, v1


def derivs6(a0, j0, s0, a1, j1, s1, dt):
    """(crackle, pop, 5th derivative) of a at the end of the step."""
    lib = _load()
    c, p, q = np.zeros(3), np.zeros(3), np.zeros(3)
    lib.or6_derivs(*(_ptr(_f64(w)) for w in (a0, j0, s0, a1, j1, s1)), float(dt), _ptr(c), _ptr(p), _ptr(q))
    return c, p, q


def aarseth6_dt(a, j, s, c, p, q, eta):
    return _load().or6_aarseth_dt(*(_ptr(_f64(w)) for w in (a, j, s, c, p, q)), float(eta))


class Sim6:
    """The time-symmetric Hermite oracle integrator: order 6 (one more
    derivative than GraviDy's scheme) or order 4 (GraviDy's scheme with the
    time-symmetric corrector), n_iter evaluation-correction passes per block
    step."""

    def __init__(self, m, x, v, eps, eta, eta_init=0.001, dt_min=2.0 ** -22, dt_max=0.125, fixed_dtau=0,
                 order=6, n_iter=1):
        self._lib = _load()
        m = _f64(m)
        self.n = n = m.shape[0]
        self.dt_min = float(dt_min)
        x = _f64(x, (n, 3))
        v = _f64(v, (n, 3))
        h = self._lib.or6_sim_new(n, _ptr(m), _ptr(x), _ptr(v), float(eps), float(eta), float(eta_init),
                                  self.dt_min, float(dt_max), int(fixed_dtau), int(order), int(n_iter))
        if not h:
            raise ValueError("oracle rejected the arguments")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or6_sim_free(h)
            self._h = None

    def step(self):
        idx = np.zeros(self.n, np.int32)
        t = ctypes.c_int64()
        c = self._lib.or6_sim_step(self._h, ctypes.byref(t), _ptr(idx))
        return t.value, idx[:c].copy()

    def replay(self, tick, idx):
        idx = np.ascontiguousarray(idx, np.int32)
        self._lib.or6_sim_replay(self._h, int(tick), idx.shape[0], _ptr(idx))

    def evolve(self, t_end):
        return self._lib.or6_sim_evolve(self._h, int(round(t_end / self.dt_min)))

    def energy(self):
        K = ctypes.c_double()
        U = ctypes.c_double()
        self._lib.or6_sim_energy(self._h, ctypes.byref(K), ctypes.byref(U))
        return K.value, U.value

    def state(self):
        n = self.n
        x, v, a, j, s, c = (np.zeros((n, 3)) for _ in range(6))
        tau = np.zeros(n, np.int64)
        dtau = np.zeros(n, np.int64)
        self._lib.or6_sim_get(self._h, *(_ptr(q) for q in (x, v, a, j, s, c, tau, dtau)))
        return dict(x=x, v=v, a=a, j=j, s=s, c=c, tau=tau, dtau=dtau)

    def stats(self):
        t, nb, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        it = ctypes.c_double()
        self._lib.or6_sim_stats(self._h, ctypes.byref(t), ctypes.byref(nb), ctypes.byref(ns), ctypes.byref(it))
        return dict(tick=t.value, nblock=nb.value, nsteps=ns.value, interactions=it.value)
