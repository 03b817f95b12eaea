"""ctypes binding of libgravidy_gb300.so (C ABI in include/gravidy.h).

Argument marshalling only: every step of the integration runs in the CUDA
kernels behind the ABI.  The module-level functions carry the C names
(gd_init, gd_evolve, gd_step_block, gd_energy, gd_get_state, ...);
``Integrator`` wraps a context with the same operations.  Host arrays are numpy
float64 of shape (n, 3) for vectors and (n,) for masses; times are ticks of
dt_min for the hooks.  A missing or unloadable library raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GD_OK, GD_EINVAL, GD_ENOMEM, GD_ECUDA, GD_ENONFINITE, GD_ETIMEOUT, GD_ESTATE = 0, -1, -2, -3, -4, -5, -6
GD_FP64, GD_MIXED = 0, 1
GD_CORR_HERMITE, GD_CORR_TIMESYM = 0, 1
GD_PN_1, GD_PN_2, GD_PN_25 = 1, 2, 4
_PRECISION = {"fp64": GD_FP64, "mixed": GD_MIXED, GD_FP64: GD_FP64, GD_MIXED: GD_MIXED}

# every entry point the header declares
EXPORTS = (
    "gd_opts_default", "gd_init", "gd_evolve", "gd_step_block", "gd_energy", "gd_get_state",
    "gd_set_state", "gd_get_stats", "gd_kernel_time", "gd_free", "gd_last_error", "gd_force",
    "gd_predict", "gd_predict_records", "gd_step_block_small", "gd_active", "gd_replay_step", "gd_test_wait_timeout", "gd_test_fail_alloc", "gd_probe_fma", "gd_force_noalloc", "gd_autotune", "gd_get_tuning", "gd_set_tuning",
    "gd_cluster_info", "gd_cluster_time", "gd_cluster_phases",
    "gd_ens_init", "gd_ens_evolve", "gd_ens_step_block", "gd_ens_energy", "gd_ens_get_state",
    "gd_ens_get_stats", "gd_ens_free", "gd_ens_last_error",
    "gd_h6_init", "gd_h6_init_scheme", "gd_h6_evolve", "gd_h6_step_block", "gd_h6_replay_step", "gd_h6_force", "gd_h6_energy",
    "gd_h6_get_state", "gd_h6_get_stats", "gd_h6_free", "gd_h6_last_error",
)


class GravidyError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


class gd_opts(ctypes.Structure):
    _fields_ = [
        ("dt_min", ctypes.c_double),
        ("dt_max", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("use_graph", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("jsplit", ctypes.c_int32),
        ("mode_cut", ctypes.c_int32),
        ("time_force", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("fused", ctypes.c_int32),
        ("pdl", ctypes.c_int32),
        ("tail_correct", ctypes.c_int32),
        ("cluster", ctypes.c_int32),
        ("corrector", ctypes.c_int32),
        ("pn_terms", ctypes.c_int32),
        ("pn_p", ctypes.c_int32),
        ("pn_q", ctypes.c_int32),
        ("pn_c", ctypes.c_double),
        ("n_iter", ctypes.c_int32),
    ]


class gd_stats(ctypes.Structure):
    _fields_ = [
        ("tick", ctypes.c_int64),
        ("block_steps", ctypes.c_int64),
        ("particle_steps", ctypes.c_int64),
        ("interactions", ctypes.c_double),
        ("last_nact", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("phase_ms", ctypes.c_double * 3),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first when allowed).  Raises if it
    cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise GravidyError(GD_ESTATE, "libgravidy_gb300.so is not built (%s)" % _build.LIB)
        lib = ctypes.CDLL(_build.LIB)
        P, I64, D, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32
        sig = {
            "gd_opts_default": (None, [P]),
            "gd_init": (ctypes.c_int, [P, I64, P, P, P, D, D, P]),
            "gd_evolve": (ctypes.c_int, [P, D]),
            "gd_step_block": (ctypes.c_int, [P, P, P]),
            "gd_energy": (ctypes.c_int, [P, P, P]),
            "gd_get_state": (ctypes.c_int, [P, P, P, P, P, P, P]),
            "gd_set_state": (ctypes.c_int, [P, P, P, P, P, P, P]),
            "gd_get_stats": (ctypes.c_int, [P, P]),
            "gd_kernel_time": (ctypes.c_int, [P, P, P, P]),
            "gd_cluster_info": (ctypes.c_int, [P, P, P, P]),
            "gd_cluster_time": (ctypes.c_int, [P, P, P]),
            "gd_cluster_phases": (ctypes.c_int, [P, P, I32, P]),
            "gd_free": (None, [P]),
            "gd_last_error": (ctypes.c_char_p, [P]),
            "gd_force": (ctypes.c_int, [P, I64, P, I64, P, P]),
            "gd_predict": (ctypes.c_int, [P, I64, P, P]),
            "gd_predict_records": (ctypes.c_int, [P, I64, P, P]),
            "gd_step_block_small": (ctypes.c_int, [P, P, P]),
            "gd_active": (ctypes.c_int, [P, P, P, P]),
            "gd_replay_step": (ctypes.c_int, [P, I64, P, I64]),
            "gd_test_wait_timeout": (ctypes.c_int, [P, I32]),
            "gd_test_fail_alloc": (ctypes.c_int, [I32, I32]),
            "gd_probe_fma": (ctypes.c_int, [I32, I32, P, P]),
            "gd_force_noalloc": (ctypes.c_int, [I64, P, P, P, D, P, I64, P, P, P]),
            "gd_autotune": (ctypes.c_int, [P, I32]),
            "gd_get_tuning": (ctypes.c_int, [P, P, P, P, P, I32]),
            "gd_set_tuning": (ctypes.c_int, [P, I32, P, P, I32]),
            "gd_ens_init": (ctypes.c_int, [P, I32, P, P, P, P, D, D, P]),
            "gd_ens_evolve": (ctypes.c_int, [P, D]),
            "gd_ens_step_block": (ctypes.c_int, [P, P, P]),
            "gd_ens_energy": (ctypes.c_int, [P, P, P]),
            "gd_ens_get_state": (ctypes.c_int, [P, P, P, P, P]),
            "gd_ens_get_stats": (ctypes.c_int, [P, P]),
            "gd_ens_free": (None, [P]),
            "gd_ens_last_error": (ctypes.c_char_p, [P]),
            "gd_h6_init": (ctypes.c_int, [P, I64, P, P, P, D, D, D, P]),
            "gd_h6_init_scheme": (ctypes.c_int, [P, I64, P, P, P, D, D, D, I32, I32, P]),
            "gd_h6_evolve": (ctypes.c_int, [P, D]),
            "gd_h6_step_block": (ctypes.c_int, [P, P, P]),
            "gd_h6_replay_step": (ctypes.c_int, [P, I64, P, I64]),
            "gd_h6_force": (ctypes.c_int, [P, I64, P, I64, P, P, P]),
            "gd_h6_energy": (ctypes.c_int, [P, P, P]),
            "gd_h6_get_state": (ctypes.c_int, [P, P, P, P, P, P, P, P, P]),
            "gd_h6_get_stats": (ctypes.c_int, [P, P]),
            "gd_h6_free": (None, [P]),
            "gd_h6_last_error": (ctypes.c_char_p, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, ctx=None):
    if rc != GD_OK:
        msg = load().gd_last_error(ctx)
        raise GravidyError(rc, msg.decode() if msg else "error")


def make_opts(dt_min=2.0 ** -22, dt_max=0.125, precision="mixed", device=0, stream=None, use_graph=True,
              graph_steps=16, jsplit=0, mode_cut=0, time_force=False, autotune=False, fused=False, pdl=None,
              tail_correct=None, cluster=None, corrector="hermite", pn=None, n_iter=1):
    o = gd_opts()
    load().gd_opts_default(ctypes.byref(o))
    o.dt_min = float(dt_min)
    o.dt_max = float(dt_max)
    o.precision = _PRECISION[precision]
    o.device = int(device)
    o.stream = stream
    o.use_graph = 1 if use_graph else 0
    o.graph_steps = int(graph_steps)
    o.jsplit = int(jsplit)
    o.mode_cut = int(mode_cut)
    o.time_force = 1 if time_force else 0
    o.autotune = 1 if autotune else 0
    o.fused = 1 if fused else 0
    if pdl is not None:
        o.pdl = 1 if pdl else 0
    if tail_correct is not None:
        o.tail_correct = 1 if tail_correct else 0
    if cluster is not None:
        o.cluster = 1 if cluster else 0
    o.corrector = {"hermite": GD_CORR_HERMITE, "timesym": GD_CORR_TIMESYM}[corrector]
    if pn is not None:  # (p, q, c, terms)
        o.pn_p, o.pn_q, o.pn_c, o.pn_terms = int(pn[0]), int(pn[1]), float(pn[2]), int(pn[3])
    o.n_iter = int(n_iter)
    return o


# ---- module-level functions with the C names -------------------------------

def gd_init(m, x, v, eps, eta, **opts):
    lib = load()
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float64))
    n = m.shape[0]
    x = _f64(x, (n, 3))
    v = _f64(v, (n, 3))
    o = make_opts(**opts)
    h = ctypes.c_void_p()
    _check(lib.gd_init(ctypes.byref(h), n, _p(m), _p(x), _p(v), float(eps), float(eta), ctypes.byref(o)))
    return h


def gd_evolve(ctx, t_end):
    _check(load().gd_evolve(ctx, float(t_end)), ctx)


def gd_step_block(ctx):
    t = ctypes.c_double()
    k = ctypes.c_int64()
    _check(load().gd_step_block(ctx, ctypes.byref(t), ctypes.byref(k)), ctx)
    return t.value, k.value


def gd_step_block_small(ctx):
    t = ctypes.c_double()
    k = ctypes.c_int64()
    _check(load().gd_step_block_small(ctx, ctypes.byref(t), ctypes.byref(k)), ctx)
    return t.value, k.value


def gd_energy(ctx):
    K = ctypes.c_double()
    U = ctypes.c_double()
    _check(load().gd_energy(ctx, ctypes.byref(K), ctypes.byref(U)), ctx)
    return K.value, U.value


def gd_get_state(ctx, n, out=None):
    """dict of x, v, a, j (n, 3) and tau, dtau (n,) int64; ``out`` may supply
    preallocated (e.g. pinned) arrays with those keys."""
    o = out if out is not None else {}
    for k in ("x", "v", "a", "j"):
        if k not in o:
            o[k] = np.empty((n, 3))
    for k in ("tau", "dtau"):
        if k not in o:
            o[k] = np.empty(n, np.int64)
    _check(load().gd_get_state(ctx, _p(o["x"]), _p(o["v"]), _p(o["a"]), _p(o["j"]), _p(o["tau"]), _p(o["dtau"])), ctx)
    return o


def gd_set_state(ctx, n, x, v, a, j, tau, dtau):
    x, v, a, j = (_f64(q, (n, 3)) for q in (x, v, a, j))
    tau = np.ascontiguousarray(tau, dtype=np.int64)
    dtau = np.ascontiguousarray(dtau, dtype=np.int64)
    _check(load().gd_set_state(ctx, _p(x), _p(v), _p(a), _p(j), _p(tau), _p(dtau)), ctx)


def gd_get_stats(ctx):
    s = gd_stats()
    _check(load().gd_get_stats(ctx, ctypes.byref(s)), ctx)
    return dict(tick=s.tick, block_steps=s.block_steps, particle_steps=s.particle_steps,
                interactions=s.interactions, last_nact=s.last_nact, kernel_launches=s.kernel_launches,
                phase_ms=list(s.phase_ms))


def gd_kernel_time(ctx):
    """(milliseconds, launches, interactions) of the timed force launches."""
    ms = ctypes.c_double()
    k = ctypes.c_int64()
    it = ctypes.c_double()
    _check(load().gd_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(k), ctypes.byref(it)), ctx)
    return ms.value, k.value, it.value


def gd_cluster_info(ctx):
    """(CTAs per cluster or 0, particles per CTA, largest cluster step) of gd_evolve."""
    cs = ctypes.c_int32()
    pc = ctypes.c_int32()
    mx = ctypes.c_int32()
    _check(load().gd_cluster_info(ctx, ctypes.byref(cs), ctypes.byref(pc), ctypes.byref(mx)), ctx)
    return cs.value, pc.value, mx.value


def gd_cluster_time(ctx):
    """(milliseconds, launches) of the timed small-step cluster launches."""
    ms = ctypes.c_double()
    k = ctypes.c_int64()
    _check(load().gd_cluster_time(ctx, ctypes.byref(ms), ctypes.byref(k)), ctx)
    return ms.value, k.value


def gd_cluster_phases(ctx):
    """(cycles[12], max SM clock kHz) of the small-step cluster's phase counters."""
    cyc = np.zeros(12)
    khz = ctypes.c_int32()
    _check(load().gd_cluster_phases(ctx, _p(cyc), 12, ctypes.byref(khz)), ctx)
    return cyc, khz.value


def gd_autotune(ctx, reps=3):
    _check(load().gd_autotune(ctx, int(reps)), ctx)


def gd_get_tuning(ctx):
    """(mode_cut, split[32], mode[32], ms[32]) of the force-kernel tuning table."""
    mc = ctypes.c_int32()
    split = np.zeros(32, np.int16)
    mode = np.zeros(32, np.int8)
    ms = np.zeros(32, np.float32)
    _check(load().gd_get_tuning(ctx, ctypes.byref(mc), _p(split), _p(mode), _p(ms), 32), ctx)
    return mc.value, split, mode, ms


def gd_set_tuning(ctx, mode_cut, split, mode):
    split = np.ascontiguousarray(split, np.int16)
    mode = np.ascontiguousarray(mode, np.int8)
    nb = min(split.size, mode.size, 32)
    _check(load().gd_set_tuning(ctx, int(mode_cut), _p(split), _p(mode), nb), ctx)


def gd_free(ctx):
    if ctx is not None and ctx.value:
        load().gd_free(ctx)


def gd_force(ctx, tick, idx):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    k = idx.shape[0]
    acc = np.empty((k, 3))
    jrk = np.empty((k, 3))
    _check(load().gd_force(ctx, int(tick), _p(idx), k, _p(acc), _p(jrk)), ctx)
    return acc, jrk


def gd_predict(ctx, n, tick):
    xp = np.empty((n, 3))
    vp = np.empty((n, 3))
    _check(load().gd_predict(ctx, int(tick), _p(xp), _p(vp)), ctx)
    return xp, vp


def gd_predict_records(ctx, n, tick):
    xp = np.empty((n, 3))
    vp = np.empty((n, 3))
    _check(load().gd_predict_records(ctx, int(tick), _p(xp), _p(vp)), ctx)
    return xp, vp


def gd_active(ctx, n):
    idx = np.empty(n, np.int32)
    k = ctypes.c_int64()
    t = ctypes.c_int64()
    _check(load().gd_active(ctx, _p(idx), ctypes.byref(k), ctypes.byref(t)), ctx)
    return idx[: k.value].copy(), t.value


def gd_replay_step(ctx, tick, idx):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    _check(load().gd_replay_step(ctx, int(tick), _p(idx), idx.shape[0]), ctx)


def gd_test_fail_alloc(kind, nth):
    """Make the nth host (kind 0) or device (kind 1) allocation of the calling
    thread's next context set-ups fail once (nth = 0 cancels)."""
    rc = load().gd_test_fail_alloc(int(kind), int(nth))
    _check(rc)


def gd_probe_fma(device=0, iters=1 << 16):
    """(TFLOP/s, ms) of the FP32 FMA throughput probe."""
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load().gd_probe_fma(int(device), int(iters), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def gd_force_noalloc(n, m_ptr, x_ptr, v_ptr, eps, idx_ptr, nact, acc_ptr, jerk_ptr, stream=None):
    """Allocation-free force/jerk evaluation on caller-owned device buffers
    (raw device addresses as ints); queues the work on ``stream`` and returns."""
    rc = load().gd_force_noalloc(int(n), m_ptr, x_ptr, v_ptr, float(eps), idx_ptr, int(nact), acc_ptr, jerk_ptr,
                                 stream)
    _check(rc)


class Integrator:
    """One gd_ctx: the GPU Hermite-4 block-step integrator."""

    def __init__(self, m, x, v, eps, eta, **opts):
        self.n = int(np.asarray(m).shape[0])
        self.dt_min = float(opts.get("dt_min", 2.0 ** -22))
        self.dt_max = float(opts.get("dt_max", 0.125))
        self._h = gd_init(m, x, v, eps, eta, **opts)

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None:
            gd_free(h)

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def evolve(self, t_end):
        gd_evolve(self._h, t_end)

    def step_block(self):
        return gd_step_block(self._h)

    def energy(self):
        return gd_energy(self._h)

    def state(self, out=None):
        return gd_get_state(self._h, self.n, out)

    def set_state(self, x, v, a, j, tau, dtau):
        gd_set_state(self._h, self.n, x, v, a, j, tau, dtau)

    def stats(self):
        return gd_get_stats(self._h)

    def kernel_time(self):
        return gd_kernel_time(self._h)

    def autotune(self, reps=3):
        gd_autotune(self._h, reps)

    def cluster_info(self):
        return gd_cluster_info(self._h)

    def cluster_phases(self):
        return gd_cluster_phases(self._h)

    def cluster_time(self):
        return gd_cluster_time(self._h)

    def set_tuning(self, mode_cut, split, mode):
        gd_set_tuning(self._h, mode_cut, split, mode)

    def tuning(self):
        return gd_get_tuning(self._h)

    def force(self, tick, idx):
        return gd_force(self._h, tick, idx)

    def predict(self, tick):
        return gd_predict(self._h, self.n, tick)

    def step_block_small(self):
        return gd_step_block_small(self._h)

    def predict_records(self, tick):
        return gd_predict_records(self._h, self.n, tick)

    def active(self):
        return gd_active(self._h, self.n)

    def replay_step(self, tick, idx):
        gd_replay_step(self._h, tick, idx)


def _check_ens(rc, h=None):
    if rc != GD_OK:
        msg = load().gd_ens_last_error(h)
        raise GravidyError(rc, msg.decode() if msg else "error")


class Ensemble:
    """gd_ens: independent clusters advanced together (mixed precision)."""

    def __init__(self, sizes, m, x, v, eps, eta, **opts):
        lib = load()
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        self.sizes = sizes
        self.C = int(sizes.size)
        self.n = int(sizes.sum())
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64))
        x = _f64(x, (self.n, 3))
        v = _f64(v, (self.n, 3))
        opts.setdefault("precision", "mixed")
        o = make_opts(**opts)
        self.dt_min = o.dt_min
        h = ctypes.c_void_p()
        _check_ens(lib.gd_ens_init(ctypes.byref(h), self.C, _p(sizes), _p(m), _p(x), _p(v), float(eps), float(eta),
                                   ctypes.byref(o)))
        self._h = h

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            load().gd_ens_free(h)

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def evolve(self, t_end):
        _check_ens(load().gd_ens_evolve(self._h, float(t_end)), self._h)

    def step_block(self):
        t = ctypes.c_double()
        k = ctypes.c_int64()
        _check_ens(load().gd_ens_step_block(self._h, ctypes.byref(t), ctypes.byref(k)), self._h)
        return t.value, k.value

    def energy(self):
        K = np.empty(self.C)
        U = np.empty(self.C)
        _check_ens(load().gd_ens_energy(self._h, _p(K), _p(U)), self._h)
        return K, U

    def state(self):
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        tau = np.empty(self.n, np.int64)
        dtau = np.empty(self.n, np.int64)
        _check_ens(load().gd_ens_get_state(self._h, _p(x), _p(v), _p(tau), _p(dtau)), self._h)
        return dict(x=x, v=v, tau=tau, dtau=dtau)

    def stats(self):
        s = gd_stats()
        _check_ens(load().gd_ens_get_stats(self._h, ctypes.byref(s)), self._h)
        return dict(tick=s.tick, block_steps=s.block_steps, particle_steps=s.particle_steps,
                    interactions=s.interactions, last_nact=s.last_nact, kernel_launches=s.kernel_launches)


def _check_h6(rc, h=None):
    if rc != GD_OK:
        msg = load().gd_h6_last_error(h)
        raise GravidyError(rc, msg.decode() if msg else "error")


class Integrator6:
    """gd_h6: the time-symmetric Hermite block-step integrators (FP64): order 6
    (sixth-order Hermite) or order 4 (the fourth-order scheme with the
    time-symmetric corrector), n_iter evaluation-correction passes per step."""

    def __init__(self, m, x, v, eps, eta, eta_init=0.001, order=6, n_iter=1, **opts):
        lib = load()
        m = np.ascontiguousarray(np.asarray(m, dtype=np.float64))
        self.n = n = m.shape[0]
        x = _f64(x, (n, 3))
        v = _f64(v, (n, 3))
        opts.setdefault("precision", "fp64")
        o = make_opts(**opts)
        self.dt_min = o.dt_min
        h = ctypes.c_void_p()
        _check_h6(lib.gd_h6_init_scheme(ctypes.byref(h), n, _p(m), _p(x), _p(v), float(eps), float(eta),
                                        float(eta_init), int(order), int(n_iter), ctypes.byref(o)))
        self._h = h

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None:
            load().gd_h6_free(h)

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def evolve(self, t_end):
        _check_h6(load().gd_h6_evolve(self._h, float(t_end)), self._h)

    def step_block(self):
        t = ctypes.c_double()
        k = ctypes.c_int64()
        _check_h6(load().gd_h6_step_block(self._h, ctypes.byref(t), ctypes.byref(k)), self._h)
        return t.value, k.value

    def replay_step(self, tick, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        _check_h6(load().gd_h6_replay_step(self._h, int(tick), _p(idx), idx.shape[0]), self._h)

    def force(self, tick, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        k = idx.shape[0]
        acc, jrk, snp = np.empty((k, 3)), np.empty((k, 3)), np.empty((k, 3))
        _check_h6(load().gd_h6_force(self._h, int(tick), _p(idx), k, _p(acc), _p(jrk), _p(snp)), self._h)
        return acc, jrk, snp

    def energy(self):
        K = ctypes.c_double()
        U = ctypes.c_double()
        _check_h6(load().gd_h6_energy(self._h, ctypes.byref(K), ctypes.byref(U)), self._h)
        return K.value, U.value

    def state(self):
        n = self.n
        o = {k: np.empty((n, 3)) for k in ("x", "v", "a", "j", "s", "c")}
        o["tau"] = np.empty(n, np.int64)
        o["dtau"] = np.empty(n, np.int64)
        _check_h6(load().gd_h6_get_state(self._h, *(_p(o[k]) for k in ("x", "v", "a", "j", "s", "c", "tau", "dtau"))),
                  self._h)
        return o

    def stats(self):
        st = gd_stats()
        _check_h6(load().gd_h6_get_stats(self._h, ctypes.byref(st)), self._h)
        return dict(tick=st.tick, block_steps=st.block_steps, particle_steps=st.particle_steps,
                    interactions=st.interactions, last_nact=st.last_nact, kernel_launches=st.kernel_launches)
