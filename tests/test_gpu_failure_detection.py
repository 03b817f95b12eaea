"""Failure detection on the GPU without a fault: a bounded device wait that
runs out (a counter that nothing advances) records GD_ETIMEOUT in the device
flag; the host reads it at the next synchronisation and returns it, the
context then refuses further work, and the GPU stays usable for a new
context (its forces still match the oracle)."""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS, ETA = 1e-4, 0.01


def test_bounded_wait_runs_out_and_is_reported():
    lib = gravidy.load()
    m, x, v = inputs.plummer(256, seed=1)
    g = gravidy.Integrator(m, x, v, EPS, ETA)
    try:
        # a limit out of range is refused on the host and leaves the context usable
        assert lib.gd_test_wait_timeout(g.handle, 0) == gravidy.GD_EINVAL
        K0, U0 = g.energy()
        # the wait gives up after 4096 polls
        assert lib.gd_test_wait_timeout(g.handle, 4096) == gravidy.GD_ETIMEOUT
        assert "wait" in lib.gd_last_error(g.handle).decode()
        with pytest.raises(gravidy.GravidyError) as e:
            g.evolve(0.125)
        assert e.value.code == gravidy.GD_ETIMEOUT
    finally:
        g.close()
    # the CUDA context and the GPU are fine: a new context works
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g2:
        idx = np.arange(256, dtype=np.int32)
        acc, jerk = g2.force(0, idx)
        K1, U1 = g2.energy()
    a, j = oracle.force(m, x, v, EPS)
    assert np.abs(acc - a).max() <= 1e-12 * np.abs(a).max()
    assert abs((K1 + U1) - (K0 + U0)) <= 1e-6 * abs(K0 + U0)


@pytest.mark.parametrize("entry", ["single", "h6", "ensemble"])
def test_injected_device_allocation_failures_return_enomem_without_leaks(entry):
    """Every device allocation of a context's set-up, made to fail in turn
    (gd_test_fail_alloc), is reported as GD_ENOMEM; the set-up frees what it
    had allocated (device memory returns to its level before), and the next
    set-up succeeds."""
    torch = pytest.importorskip("torch")
    n = 100000  # planes of 2.4 MB, so a leaked allocation shows in the free memory
    m, x, v = inputs.plummer(n, seed=3)

    def make():
        if entry == "single":
            return gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", cluster=False)
        if entry == "h6":
            return gravidy.Integrator6(m, x, v, EPS, ETA)
        return gravidy.Ensemble([n // 2, n - n // 2], m, x, v, EPS, ETA)

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 64):
        gravidy.gd_test_fail_alloc(1, k)
        try:
            g = make()
        except gravidy.GravidyError as e:
            assert e.code == gravidy.GD_ENOMEM
            failures += 1
            continue
        # k is beyond the set-up's allocations: it succeeded; cancel and stop
        gravidy.gd_test_fail_alloc(1, 0)
        g.close()
        break
    assert failures >= 5
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= 8 << 20, (free0, free1)
