"""gd_force_noalloc, the allocation-free force entry point, against gd_force.

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
# the mixed-precision bound of the other GPU tests: per component, 160 units of
# 2^-24 times the sum of the term magnitudes; two such results differ by at most twice that
MIXED_TERM_BOUND = 160 * 2.0 ** -24


def _dev(a, torch, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_no_alloc_force_matches_gd_force_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    gravidy.load()
    oracle.build()
    n = 5000
    m, x, v = inputs.plummer(n, seed=21, masses=inputs.power_law_masses(n, seed=21))
    dm, dx, dv = _dev(m, torch, torch.float64), _dev(x, torch, torch.float64), _dev(v, torch, torch.float64)
    stream = torch.cuda.Stream()
    # two calls in a row: a small active set (warp mode, j-split) then every particle
    for idx in (inputs.random_subset(n, 37, seed=3), np.arange(n, dtype=np.int32)):
        k = idx.size
        didx = _dev(idx, torch, torch.int32)
        acc = torch.full((k, 3), float("nan"), dtype=torch.float64, device="cuda")
        jrk = torch.full((k, 3), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        gravidy.gd_force_noalloc(n, dm.data_ptr(), dx.data_ptr(), dv.data_ptr(), EPS, didx.data_ptr(), k,
                                 acc.data_ptr(), jrk.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        a_new, j_new = acc.cpu().numpy(), jrk.cpu().numpy()
        with gravidy.Integrator(m, x, v, EPS, 0.01, precision="mixed") as g:
            a_ref, j_ref = g.force(0, idx)
        an, jn = oracle.force_absnorm(m, x, v, EPS, idx)
        assert np.all(np.isfinite(a_new)) and np.all(np.isfinite(j_new))
        assert (np.abs(a_new - a_ref).max(axis=1) <= 2 * MIXED_TERM_BOUND * an).all()
        assert (np.abs(j_new - j_ref).max(axis=1) <= 2 * MIXED_TERM_BOUND * jn).all()


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    gravidy.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(gravidy.GravidyError) as e:
        gravidy.gd_force_noalloc(32769, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), EPS, buf.data_ptr(), 1,
                                 buf.data_ptr(), buf.data_ptr(), None)
    assert e.value.code == gravidy.GD_EINVAL
    assert "32768" in str(e.value)
