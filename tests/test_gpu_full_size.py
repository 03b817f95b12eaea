"""Full-size cases on the GPU, checked on outputs the oracle can compute one by
one, and on properties that hold at any size.

- Plummer N = 2^20, force of random active sets of 1, 32, 1024, 32768 and all
  2^20 particles (mixed), 1..32768 (FP64): 48 sampled slots vs the oracle.
- Plummer N = 16384 integrated in mixed precision; at 64 random block times the
  force of 32 random particles from both GPU paths vs the oracle on the
  oracle's own prediction of the state.
- Plummer N = 262144 with power-law masses (dN/dm ~ m^-2.35 on [0.2, 20]):
  sampled forces, Newton's third law over the full evaluation, and block-step
  invariants over a stretch of integration.
Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
ETA = 0.01
DT_MIN = 2.0 ** -22
U32 = 2.0 ** -24
MIXED_TERM_BOUND = 160 * U32


def fp64_term_bound(n):
    """FP64 path: sums of up to n terms, each with a few ulp of its own error;
    the summation error of n terms with independent roundings stays below about
    8 sqrt(n) units with overwhelming probability (probabilistic bound of Higham
    and Mary for recursive summation), plus the per-term part."""
    return (16 + 8 * n ** 0.5) * 2.0 ** -53


@pytest.fixture(scope="module")
def big():
    gravidy.load()
    oracle.build()
    return inputs.plummer(1 << 20, seed=1)


@pytest.fixture(scope="module")
def big_ctx(big):
    """One context per precision at N = 2^20 (the FP64 one's initial full
    evaluation alone takes over a minute on this GPU's FP64 units)."""
    m, x, v = big
    ctx = {p: gravidy.Integrator(m, x, v, EPS, ETA, precision=p) for p in ("mixed", "fp64")}
    yield ctx
    for g in ctx.values():
        g.close()


def _sampled_check(m, x, v, idx, a, j, prec, nsample, seed):
    rng = np.random.default_rng(seed)
    pick = rng.choice(idx.size, size=min(nsample, idx.size), replace=False)
    sub = idx[pick]
    a_or, j_or = oracle.force(m, x, v, EPS, sub)
    an, jn = oracle.force_absnorm(m, x, v, EPS, sub)
    bound = MIXED_TERM_BOUND if prec == "mixed" else fp64_term_bound(m.size)
    ra = np.abs(a[pick] - a_or).max(axis=1) / an
    rj = np.abs(j[pick] - j_or).max(axis=1) / jn
    rel = np.linalg.norm(a[pick] - a_or, axis=1) / np.linalg.norm(a_or, axis=1)
    assert ra.max() <= bound and rj.max() <= bound, (ra.max(), rj.max())
    return np.median(rel)


@pytest.mark.parametrize("nact", [1, 32, 1024, 32768, 1 << 20])
def test_force_n2p20_mixed(big, big_ctx, nact):
    m, x, v = big
    n = m.size
    idx = np.arange(n, dtype=np.int32) if nact == n else inputs.random_subset(n, nact, seed=nact)
    a, j = big_ctx["mixed"].force(0, idx)
    med = _sampled_check(m, x, v, idx, a, j, "mixed", 48, nact)
    assert med <= 1e-6


@pytest.mark.parametrize("nact", [1, 32, 1024, 32768])
def test_force_n2p20_fp64(big, big_ctx, nact):
    m, x, v = big
    idx = inputs.random_subset(m.size, nact, seed=nact)
    a, j = big_ctx["fp64"].force(0, idx)
    med = _sampled_check(m, x, v, idx, a, j, "fp64", 48, nact)
    assert med <= 1e-12


def test_force_error_on_64_snapshots_n16384():
    n = 16384
    m, x, v = inputs.plummer(n, seed=1)
    rng = np.random.default_rng(64)
    stops = np.sort(rng.choice(np.arange(1, 1200), size=64, replace=False))
    errs = {"mixed": [], "fp64": []}
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g, \
            gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as h:
        done = 0
        for stop in stops:
            while done < stop:
                g.step_block()
                done += 1
            st = g.state()
            tick = g.stats()["tick"]
            h.set_state(st["x"], st["v"], st["a"], st["j"], st["tau"], st["dtau"])
            idx = np.sort(rng.choice(n, size=32, replace=False)).astype(np.int32)
            # the oracle's own prediction of every particle to the snapshot time
            xp, vp = oracle.predict_all(st["x"], st["v"], st["a"], st["j"], (tick - st["tau"]) * DT_MIN)
            a_or, j_or = oracle.force(m, xp, vp, EPS, idx)
            an, jn = oracle.force_absnorm(m, xp, vp, EPS, idx)
            for prec, ctx in (("mixed", g), ("fp64", h)):
                a, j = ctx.force(tick, idx)
                bound = MIXED_TERM_BOUND if prec == "mixed" else fp64_term_bound(m.size)
                # both sides predict in FP64 but in different operation orders: positions
                # may differ by a few ulp (~1e-15), which a term amplifies by up to
                # 3 |x| / r with r >= eps = 1e-4, so allow 3e-11 of the term sum
                assert (np.abs(a - a_or).max(axis=1) <= (bound + 3e-11) * an).all()
                assert (np.abs(j - j_or).max(axis=1) <= (bound + 3e-11) * jn).all()
                errs[prec].extend((np.linalg.norm(a - a_or, axis=1) / np.linalg.norm(a_or, axis=1)).tolist())
    for prec, e in errs.items():
        e = np.array(e)
        print("%s: %d samples, rel |da|/|a| median %.2e p99 %.2e max %.2e"
              % (prec, e.size, np.median(e), np.percentile(e, 99), e.max()))
    assert np.median(errs["mixed"]) <= 1e-6
    assert np.median(errs["fp64"]) <= 1e-12


def test_powerlaw_n262144_forces_and_invariants():
    n = 262144
    masses = inputs.power_law_masses(n, seed=3)
    m, x, v = inputs.plummer(n, seed=3, masses=masses)
    assert abs(m.sum() - 1.0) < 1e-12 and m.max() / m.min() > 50
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        idx = np.arange(n, dtype=np.int32)
        a, j = g.force(0, idx)
        _sampled_check(m, x, v, idx, a, j, "mixed", 32, 5)
        # Newton's third law over the whole evaluation (holds at any size):
        # |sum m a| <= sum m |error| <= 160 2^-24 sum_i m_i sum_j |term_ij|, the last sum
        # estimated from 256 sampled particles (times 2 for the estimate's spread)
        sample = inputs.random_subset(n, 256, seed=11)
        an_s, _ = oracle.force_absnorm(m, x, v, EPS, sample)
        scale = n * np.mean(m[sample] * an_s)
        assert np.abs((m[:, None] * a).sum(0)).max() < 2 * MIXED_TERM_BOUND * scale
        nb = 0
        for _ in range(300):
            t, nact = g.step_block()
            nb += 1
        st = g.state()
        assert (st["tau"] % st["dtau"] == 0).all()
        assert ((st["dtau"] & (st["dtau"] - 1)) == 0).all()
        assert np.isfinite(st["x"]).all() and np.isfinite(st["a"]).all()
        assert g.stats()["block_steps"] == nb
