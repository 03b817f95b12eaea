"""The C ABI without a GPU: the library builds, loads, and exports every
function include/gravidy.h declares; host-side argument checks of gd_init and
gd_h6_init reject bad input before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1702_00440_gb300 import gravidy

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gravidy.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(gd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gd_init", "gd_evolve", "gd_step_block", "gd_energy", "gd_get_state", "gd_free", "gd_last_error"):
        assert n in names


def test_library_exports_every_declared_function():
    lib = gravidy.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(gravidy.EXPORTS) == _declared()


def _init(n, m, x, v, eps=1e-4, eta=0.01, order=4, **kw):
    lib = gravidy.load()
    o = gravidy.make_opts(**kw)
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    if order == 6:
        rc = lib.gd_h6_init(ctypes.byref(h), n, p(m), p(x), p(v), eps, eta, 0.01, ctypes.byref(o))
        return rc, lib.gd_h6_last_error(None).decode()
    rc = lib.gd_init(ctypes.byref(h), n, p(m), p(x), p(v), eps, eta, ctypes.byref(o))
    return rc, lib.gd_last_error(None).decode()


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("case", ["n0", "eps", "eta", "dtmin", "dtorder", "mass", "nan"])
def test_gd_init_rejects_bad_arguments_on_the_host(case, order):
    n = 4
    m = np.full(n, 0.25)
    x = np.arange(12, dtype=float).reshape(4, 3)
    v = np.zeros((4, 3))
    kw = {}
    eps, eta = 1e-4, 0.01
    if case == "n0":
        n = 0
    elif case == "eps":
        eps = -1.0
    elif case == "eta":
        eta = 0.0
    elif case == "dtmin":
        kw["dt_min"] = 3e-7
    elif case == "dtorder":
        kw["dt_min"], kw["dt_max"] = 0.25, 0.125
    elif case == "mass":
        m[1] = -1.0
    elif case == "nan":
        x[2, 1] = np.nan
    rc, msg = _init(n, m, x, v, eps, eta, order, **kw)
    assert rc == gravidy.GD_EINVAL
    assert msg


@pytest.mark.parametrize("order,n_iter", [(5, 1), (2, 1), (4, 0), (6, 17), (6, -1)])
def test_h6_scheme_rejects_bad_order_and_passes_on_the_host(order, n_iter):
    lib = gravidy.load()
    n = 4
    m = np.full(n, 0.25)
    x = np.arange(12, dtype=float).reshape(4, 3)
    v = np.zeros((4, 3))
    h = ctypes.c_void_p()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.gd_h6_init_scheme(ctypes.byref(h), n, p(m), p(x), p(v), 1e-4, 0.01, 0.01, order, n_iter, None)
    assert rc == gravidy.GD_EINVAL
    assert not h.value
    assert lib.gd_h6_last_error(None).decode()


def test_wait_probe_rejects_a_null_context_on_the_host():
    lib = gravidy.load()
    assert lib.gd_test_wait_timeout(None, 100) == gravidy.GD_EINVAL
    assert lib.gd_last_error(None).decode()


def test_opts_defaults():
    o = gravidy.make_opts()
    assert o.dt_min == 2.0 ** -22 and o.dt_max == 0.125 and o.precision == gravidy.GD_MIXED


def _have_gpu():
    try:
        import torch
    except ImportError:
        return False
    return torch.cuda.is_available()


def _small_system():
    n = 4
    return n, np.full(n, 0.25), np.arange(12, dtype=float).reshape(4, 3), np.zeros((4, 3))


@pytest.mark.parametrize("entry", ["gd_init", "gd_h6_init", "gd_ens_init"])
def test_injected_host_allocation_failure_returns_enomem(entry):
    """A host allocation that fails during a context's set-up is reported as
    GD_ENOMEM with a message and leaves no context behind; the injection is
    one-shot, so the same call afterwards gets past that allocation (on a
    machine without a GPU it then stops at the first CUDA call instead)."""
    lib = gravidy.load()
    n, m, x, v = _small_system()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    o = gravidy.make_opts()
    sizes = np.array([n], dtype=np.int64)

    def call():
        h = ctypes.c_void_p()
        if entry == "gd_init":
            rc = lib.gd_init(ctypes.byref(h), n, p(m), p(x), p(v), 1e-4, 0.01, ctypes.byref(o))
            msg = lib.gd_last_error(None)
        elif entry == "gd_h6_init":
            rc = lib.gd_h6_init(ctypes.byref(h), n, p(m), p(x), p(v), 1e-4, 0.01, 0.001, ctypes.byref(o))
            msg = lib.gd_h6_last_error(None)
        else:
            rc = lib.gd_ens_init(ctypes.byref(h), 1, p(sizes), p(m), p(x), p(v), 1e-4, 0.01, ctypes.byref(o))
            msg = lib.gd_ens_last_error(None)
        return rc, msg.decode(), h

    gravidy.gd_test_fail_alloc(0, 1)
    rc, msg, h = call()
    assert rc == gravidy.GD_ENOMEM
    assert "allocation" in msg
    assert not h.value
    if _have_gpu():
        return
    rc, msg, h = call()
    assert rc == gravidy.GD_ECUDA and not h.value


def test_fail_alloc_hook_rejects_bad_arguments():
    lib = gravidy.load()
    assert lib.gd_test_fail_alloc(2, 1) == gravidy.GD_EINVAL
    assert lib.gd_test_fail_alloc(0, -1) == gravidy.GD_EINVAL
    assert lib.gd_test_fail_alloc(1, 0) == gravidy.GD_OK


def test_tiny_softening_is_checked_against_the_masses_on_the_host():
    """The softened self term m / eps^3 must be finite in the pair arithmetic's
    precision: eps = 1e-14 with unit masses overflows FP32 (mixed) but not FP64."""
    lib = gravidy.load()
    n, m, x, v = _small_system()
    m = np.ones(n)
    for prec, want in (("mixed", gravidy.GD_EINVAL), ("fp64", None)):
        o = gravidy.make_opts(precision=prec)
        h = ctypes.c_void_p()
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        rc = lib.gd_init(ctypes.byref(h), n, p(m), p(x), p(v), 1e-14, 0.01, ctypes.byref(o))
        if want is not None:
            assert rc == want and "eps" in lib.gd_last_error(None).decode()
        else:
            assert rc != gravidy.GD_EINVAL
            if h.value:
                lib.gd_free(h)


def test_fma_probe_rejects_bad_iteration_counts_on_the_host():
    lib = gravidy.load()
    tf = ctypes.c_double()
    assert lib.gd_probe_fma(0, 0, ctypes.byref(tf), None) == gravidy.GD_EINVAL
    assert lib.gd_probe_fma(0, (1 << 24) + 1, ctypes.byref(tf), None) == gravidy.GD_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """gd_opts and gd_stats as the C compiler lays them out (offset of every
    field and the size) equal the ctypes structures the binding passes."""
    import subprocess

    include = os.path.dirname(HEADER)
    lines = []
    for st, cls in (("gd_opts", gravidy.gd_opts), ("gd_stats", gravidy.gd_stats)):
        for name, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, name, st, name))
        lines.append('printf("%s.size %%zu\\n", sizeof(%s));' % (st, st))
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "gravidy.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", include, "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    for st, cls in (("gd_opts", gravidy.gd_opts), ("gd_stats", gravidy.gd_stats)):
        for name, _ in cls._fields_:
            assert int(got["%s.%s" % (st, name)]) == getattr(cls, name).offset, (st, name)
        assert int(got["%s.size" % st]) == ctypes.sizeof(cls), st


def test_pass_count_is_checked_on_the_host():
    """gd_opts.n_iter: 1 to 16 passes; more than one needs the time-symmetric
    corrector and takes neither a post-Newtonian pair nor the fused kernel nor an
    ensemble (rejected before any device work)."""
    lib = gravidy.load()
    n, m, x, v = _small_system()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    bad = (dict(n_iter=0), dict(n_iter=17), dict(n_iter=2), dict(n_iter=2, corrector="timesym", fused=True),
           dict(n_iter=2, corrector="timesym", pn=(0, 1, 10.0, 1)))
    for kw in bad:
        o = gravidy.make_opts(**kw)
        h = ctypes.c_void_p()
        assert lib.gd_init(ctypes.byref(h), n, p(m), p(x), p(v), 1e-4, 0.01, ctypes.byref(o)) == gravidy.GD_EINVAL, kw
        assert not h.value
    sizes = np.array([n], dtype=np.int64)
    o = gravidy.make_opts(n_iter=2, corrector="timesym")
    h = ctypes.c_void_p()
    assert lib.gd_ens_init(ctypes.byref(h), 1, p(sizes), p(m), p(x), p(v), 1e-4, 0.01,
                           ctypes.byref(o)) == gravidy.GD_EINVAL


def test_post_newtonian_pair_is_checked_on_the_host():
    lib = gravidy.load()
    n, m, x, v = _small_system()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    for pn in ((0, 0, 10.0, 1), (0, 4, 10.0, 1), (0, 1, -1.0, 1), (0, 1, 10.0, 8), (0, 1, float("nan"), 5)):
        o = gravidy.make_opts(pn=pn)
        h = ctypes.c_void_p()
        assert lib.gd_init(ctypes.byref(h), n, p(m), p(x), p(v), 1e-4, 0.01, ctypes.byref(o)) == gravidy.GD_EINVAL
        assert not h.value
    sizes = np.array([n], dtype=np.int64)
    o = gravidy.make_opts(pn=(0, 1, 10.0, 5))
    h = ctypes.c_void_p()
    assert lib.gd_ens_init(ctypes.byref(h), 1, p(sizes), p(m), p(x), p(v), 1e-4, 0.01,
                           ctypes.byref(o)) == gravidy.GD_EINVAL
