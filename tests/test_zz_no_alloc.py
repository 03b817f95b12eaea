"""gd_force_noalloc, the allocation-free force entry point, against gd_force and
the FP64 oracle.

Callers that cannot call cudaMalloc (another component owns the device memory
budget, or the path cannot afford an allocation) pass their own device buffers;
the entry point's scratch is a fixed array inside the library.  The buffers here
come from PyTorch's allocator, standing in for such a caller's memory.

This file sorts last so a run that stops at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
# the mixed-precision bound of the other GPU tests: per component, 16 units of
# 2^-24 times the sum of the term magnitudes; two such results differ by at most twice that
MIXED_TERM_BOUND = 16 * 2.0 ** -24


def _dev(a, torch, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _noalloc(torch, n, dm, dx, dv, eps, idx, stream):
    k = idx.size
    didx = _dev(idx, torch, torch.int32)
    acc = torch.full((k, 3), float("nan"), dtype=torch.float64, device="cuda")
    jrk = torch.full((k, 3), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    gravidy.gd_force_noalloc(n, dm.data_ptr(), dx.data_ptr(), dv.data_ptr(), eps, didx.data_ptr(), k,
                             acc.data_ptr(), jrk.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return acc.cpu().numpy(), jrk.cpu().numpy()


def _against_oracle(m, x, v, eps, idx, a, j, nsample=None):
    """Per component within the mixed bound of the oracle (all rows, or a
    seeded sample of them)."""
    rows = np.arange(idx.size)
    if nsample is not None and idx.size > nsample:
        rows = np.sort(np.random.default_rng(idx.size).choice(idx.size, size=nsample, replace=False))
    sub = idx[rows]
    a_or, j_or = oracle.force(m, x, v, eps, sub)
    an, jn = oracle.force_absnorm(m, x, v, eps, sub)
    assert (np.abs(a[rows] - a_or).max(axis=1) <= MIXED_TERM_BOUND * an).all()
    assert (np.abs(j[rows] - j_or).max(axis=1) <= MIXED_TERM_BOUND * jn).all()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def test_no_alloc_force_matches_gd_force_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    n = 5000
    m, x, v = inputs.plummer(n, seed=21, masses=inputs.power_law_masses(n, seed=21))
    dm, dx, dv = _dev(m, torch, torch.float64), _dev(x, torch, torch.float64), _dev(v, torch, torch.float64)
    stream = torch.cuda.Stream()
    # two calls in a row: a small active set (warp mode, j-split) then every particle
    for idx in (inputs.random_subset(n, 37, seed=3), np.arange(n, dtype=np.int32)):
        a_new, j_new = _noalloc(torch, n, dm, dx, dv, EPS, idx, stream)
        with gravidy.Integrator(m, x, v, EPS, 0.01, precision="mixed") as g:
            a_ref, j_ref = g.force(0, idx)
        an, jn = oracle.force_absnorm(m, x, v, EPS, idx)
        assert np.all(np.isfinite(a_new)) and np.all(np.isfinite(j_new))
        assert (np.abs(a_new - a_ref).max(axis=1) <= 2 * MIXED_TERM_BOUND * an).all()
        assert (np.abs(j_new - j_ref).max(axis=1) <= 2 * MIXED_TERM_BOUND * jn).all()
        _against_oracle(m, x, v, EPS, idx, a_new, j_new)


def test_no_alloc_at_its_largest_size():
    """n = 32768 with every particle active: the scratch layout and the j-split
    partial capacity at their limits."""
    torch = pytest.importorskip("torch")
    n = 32768
    m, x, v = inputs.plummer(n, seed=5)
    dm, dx, dv = _dev(m, torch, torch.float64), _dev(x, torch, torch.float64), _dev(v, torch, torch.float64)
    stream = torch.cuda.Stream()
    idx = np.arange(n, dtype=np.int32)
    a_new, j_new = _noalloc(torch, n, dm, dx, dv, EPS, idx, stream)
    with gravidy.Integrator(m, x, v, EPS, 0.01, precision="mixed") as g:
        a_ref, j_ref = g.force(0, idx)
    assert np.all(np.isfinite(a_new)) and np.all(np.isfinite(j_new))
    pick = np.random.default_rng(1).choice(n, size=512, replace=False)
    an, jn = oracle.force_absnorm(m, x, v, EPS, idx[pick])
    assert (np.abs(a_new[pick] - a_ref[pick]).max(axis=1) <= 2 * MIXED_TERM_BOUND * an).all()
    assert (np.abs(j_new[pick] - j_ref[pick]).max(axis=1) <= 2 * MIXED_TERM_BOUND * jn).all()
    _against_oracle(m, x, v, EPS, idx, a_new, j_new, nsample=256)


def test_no_alloc_unsoftened():
    """eps = 0: the unsoftened kernel instance, whose self term is masked."""
    torch = pytest.importorskip("torch")
    n = 700
    m, x, v = inputs.plummer(n, seed=3)
    dm, dx, dv = _dev(m, torch, torch.float64), _dev(x, torch, torch.float64), _dev(v, torch, torch.float64)
    stream = torch.cuda.Stream()
    idx = np.arange(n, dtype=np.int32)
    a_new, j_new = _noalloc(torch, n, dm, dx, dv, 0.0, idx, stream)
    assert np.all(np.isfinite(a_new)) and np.all(np.isfinite(j_new))
    _against_oracle(m, x, v, 0.0, idx, a_new, j_new)


def test_no_alloc_out_of_range_index_rows_are_nan():
    """An index outside [0, n) gives NaN in its own rows only; the other rows
    are what they would be without it."""
    torch = pytest.importorskip("torch")
    n = 3000
    m, x, v = inputs.plummer(n, seed=9)
    dm, dx, dv = _dev(m, torch, torch.float64), _dev(x, torch, torch.float64), _dev(v, torch, torch.float64)
    stream = torch.cuda.Stream()
    good = inputs.random_subset(n, 20, seed=4)
    idx = np.concatenate([good[:7], [-1], good[7:15], [n], good[15:]]).astype(np.int32)
    bad = np.array([7, 16])
    a_new, j_new = _noalloc(torch, n, dm, dx, dv, EPS, idx, stream)
    assert np.isnan(a_new[bad]).all() and np.isnan(j_new[bad]).all()
    ok = np.setdiff1d(np.arange(idx.size), bad)
    assert np.isfinite(a_new[ok]).all() and np.isfinite(j_new[ok]).all()
    _against_oracle(m, x, v, EPS, idx[ok], a_new[ok], j_new[ok])


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(gravidy.GravidyError) as e:
        gravidy.gd_force_noalloc(32769, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), EPS, buf.data_ptr(), 1,
                                 buf.data_ptr(), buf.data_ptr(), None)
    assert e.value.code == gravidy.GD_EINVAL
    assert "32768" in str(e.value)
