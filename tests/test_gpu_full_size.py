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
MIXED_TERM_BOUND = 16 * U32


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
    """Per component within the term-scaled bound on a seeded sample of the
    active set; returns the per-particle relative errors of a and jerk."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(idx.size, size=min(nsample, idx.size), replace=False)
    sub = idx[pick]
    a_or, j_or = oracle.force(m, x, v, EPS, sub)
    an, jn = oracle.force_absnorm(m, x, v, EPS, sub)
    bound = MIXED_TERM_BOUND if prec == "mixed" else fp64_term_bound(m.size)
    ra = np.abs(a[pick] - a_or).max(axis=1) / an
    rj = np.abs(j[pick] - j_or).max(axis=1) / jn
    rel_a = np.linalg.norm(a[pick] - a_or, axis=1) / np.linalg.norm(a_or, axis=1)
    rel_j = np.linalg.norm(j[pick] - j_or, axis=1) / np.linalg.norm(j_or, axis=1)
    print("%s n=%d nact=%d sample %d: max|da|/sum|a_j| %.2e max|dj|/sum|j_j| %.2e  rel a med %.2e p99 %.2e max "
          "%.2e  rel j med %.2e p99 %.2e max %.2e"
          % (prec, m.size, idx.size, pick.size, ra.max(), rj.max(), np.median(rel_a), np.percentile(rel_a, 99),
             rel_a.max(), np.median(rel_j), np.percentile(rel_j, 99), rel_j.max()))
    assert ra.max() <= bound and rj.max() <= bound, (ra.max(), rj.max())
    return rel_a, rel_j


@pytest.mark.parametrize("nact", [1, 32, 1024, 32768, 1 << 20])
def test_force_n2p20_mixed(big, big_ctx, nact):
    m, x, v = big
    n = m.size
    idx = np.arange(n, dtype=np.int32) if nact == n else inputs.random_subset(n, nact, seed=nact)
    a, j = big_ctx["mixed"].force(0, idx)
    rel_a, rel_j = _sampled_check(m, x, v, idx, a, j, "mixed", 256, nact)
    assert np.median(rel_a) <= 1e-6 and np.median(rel_j) <= 1e-6
    if rel_a.size >= 200:
        assert np.percentile(rel_a, 99) <= 1e-6 and np.percentile(rel_j, 99) <= 1e-6


@pytest.mark.parametrize("nact", [1, 32, 1024, 32768])
def test_force_n2p20_fp64(big, big_ctx, nact):
    m, x, v = big
    idx = inputs.random_subset(m.size, nact, seed=nact)
    a, j = big_ctx["fp64"].force(0, idx)
    rel_a, rel_j = _sampled_check(m, x, v, idx, a, j, "fp64", 48, nact)
    assert np.median(rel_a) <= 1e-12


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
                # the FP64 context predicts in FP64 in another operation order than the
                # oracle: positions may differ by a few ulp (~1e-15), which a term
                # amplifies by up to 3 |x| / r with r >= eps = 1e-4, so allow 3e-11 of the
                # term sum; the mixed context predicts in double-single (positions to
                # about 2^-48 of |x|, the same order of difference) and rounds the
                # predicted velocities to FP32, the rounding its j-records always carry
                # and part of the term bound
                assert (np.abs(a - a_or).max(axis=1) <= (bound + 3e-11) * an).all()
                assert (np.abs(j - j_or).max(axis=1) <= (bound + 3e-11) * jn).all()
                errs[prec].append((np.linalg.norm(a - a_or, axis=1) / np.linalg.norm(a_or, axis=1),
                                   np.linalg.norm(j - j_or, axis=1) / np.linalg.norm(j_or, axis=1)))
    for prec in errs:
        ea = np.concatenate([q[0] for q in errs[prec]])
        ej = np.concatenate([q[1] for q in errs[prec]])
        print("%s: %d samples, rel |da|/|a| median %.2e p99 %.2e max %.2e; |dj|/|j| median %.2e p99 %.2e max %.2e"
              % (prec, ea.size, np.median(ea), np.percentile(ea, 99), ea.max(), np.median(ej),
                 np.percentile(ej, 99), ej.max()))
        tol = 1e-6 if prec == "mixed" else 1e-12
        assert np.median(ea) <= tol and np.median(ej) <= tol
        assert np.percentile(ea, 99) <= tol and np.percentile(ej, 99) <= tol


def test_powerlaw_n262144_forces_and_invariants():
    n = 262144
    masses = inputs.power_law_masses(n, seed=3)
    m, x, v = inputs.plummer(n, seed=3, masses=masses)
    assert abs(m.sum() - 1.0) < 1e-12 and m.max() / m.min() > 50
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        idx = np.arange(n, dtype=np.int32)
        a, j = g.force(0, idx)
        rel_a, rel_j = _sampled_check(m, x, v, idx, a, j, "mixed", 256, 5)
        # power-law masses: the jerk's tail of cancelling sums is longer than for equal masses
        assert np.percentile(rel_a, 99) <= 1e-6 and np.percentile(rel_j, 99) <= 1.5e-6
        # Newton's third law over the whole evaluation (holds at any size):
        # |sum m a| <= sum m |error| <= 16 2^-24 sum_i m_i sum_j |term_ij|, the last sum
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
