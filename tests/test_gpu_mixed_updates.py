"""The mixed path's prediction and correction element by element against the
oracle, from identical inputs.

The mixed path keeps positions and velocities as double-single values (hi + lo
floats, about 48 significant bits) and accelerations and jerks as FP32, and
predicts (Sec. 2.4 step 7a), corrects (step 7d) and chooses the new block step
(Aarseth's criterion, Sec. 3.2) with FP32 instructions.  The oracle does the same
steps in FP64 on the same input values (the state read back from the GPU is the
exact value of its double-single / FP32 representation), so the differences
are the mixed path's own rounding, bounded below from its arithmetic:

predictor (double-single position of the j-record, FP32 velocity)
  x: the exact product dt*v.hi plus a handful of FP32 roundings of terms no
     larger than 2^-24 |x| + |v dt| (the lo parts and the product residual),
     plus FP32 roundings of the a dt^2/2 + jerk dt^3/6 terms (h3 carries the
     rounding of 1/6):  |dx| <= 8 2^-48 (|x| + 2 |v dt|) + 8 2^-24 (|a| dt^2/2 + |j| dt^3/6)
  v: the record's velocity is the FP32 rounding of the predicted one (half an
     ulp, at most 2^-24 of it) plus FP32 roundings of the a dt + jerk dt^2/2 terms:
     |dv| <= 2^-24 |v_p| + 4 2^-24 (|a| dt + |j| dt^2/2) + 2^-44 |v|
corrector (FP32 Hermite derivatives from FP32 end-point forces)
  a2 dt^2 = -6 (a0 - a1) - dt (4 j0 + 2 j1) and a3 dt^3 = 12 (a0 - a1) + 6 dt (j0 + j1)
  are FP32 sums of terms bounded by S2 = 6|a0 - a1| + dt (4|j0| + 2|j1|) and
  S3 = 12|a0 - a1| + 6 dt (|j0| + |j1|), each rounded a few times; the corrections
  a2 dt^4/24 + a3 dt^5/120 (x) and a2 dt^3/6 + a3 dt^4/24 (v) then carry
  |dx| <= pred + 8 2^-24 (S2/24 + S3/120) dt^2 + 4 2^-48 |x|,
  |dv| <= 4 2^-48 |v| + 4 2^-24 (|a0| dt + |j0| dt^2/2) + 8 2^-24 (S2/6 + S3/24) dt.
new block step: the same power-of-two rules; the FP32 norms and the rounding of
  a2 and a3 above move the estimate by a relative amount r bounded from the same
  sums, so the mixed and FP64 decisions may differ only where the oracle's
  estimate lies within a factor (1 + 4 r) of a decision boundary (a power of two
  times dt_min).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS, ETA = 1e-4, 0.01
DT_MIN = 2.0 ** -22
DTAU_MAX = int(0.125 / DT_MIN)
U24, U48, U53 = 2.0 ** -24, 2.0 ** -48, 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def _pred_bounds(x, v, a, j, vo, dt):
    bx = 8 * U48 * (np.abs(x) + 2 * np.abs(v * dt)) + 8 * U24 * (np.abs(a) * dt * dt / 2 + np.abs(j) * dt ** 3 / 6) \
        + 4 * U53 * (np.abs(x) + np.abs(v * dt))
    bv = U24 * np.abs(vo) + 4 * U24 * (np.abs(a) * dt + np.abs(j) * dt * dt / 2) + 2.0 ** -44 * np.abs(v)
    return bx, bv


@pytest.mark.parametrize("ahead", [0, 2048, 65536])
def test_mixed_predictor_matches_oracle_elementwise(ahead):
    """Every particle of an integrated N = 3000 system, predicted to the block
    time of the last step plus `ahead` ticks (up to 1/64 N-body units)."""
    n = 3000
    m, x, v = inputs.plummer(n, seed=31)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        g.evolve(0.125)
        for _ in range(25):
            g.step_block()
        st = g.state()
        tick = g.stats()["tick"] + ahead
        xp, vp = g.predict_records(tick)
    dt = (tick - st["tau"]) * DT_MIN
    assert (dt >= 0).all() and dt.max() > 0
    worst_x = worst_v = 0.0
    for i in range(n):
        xo, vo = oracle.predict_one(st["x"][i], st["v"][i], st["a"][i], st["j"][i], dt[i])
        bx, bv = _pred_bounds(st["x"][i], st["v"][i], st["a"][i], st["j"][i], vo, dt[i])
        ex, ev = np.abs(xp[i] - xo), np.abs(vp[i] - vo)
        assert (ex <= bx).all(), (i, ex, bx)
        assert (ev <= bv).all(), (i, ev, bv)
        worst_x = max(worst_x, float((ex / bx).max()))
        worst_v = max(worst_v, float((ev / bv).max()))
    print("predictor ahead=%d: worst |dx|/bound %.3f, |dv|/bound %.3f" % (ahead, worst_x, worst_v))


def _near_boundary(dt_new, rel):
    """True if dt_new lies within a factor (1 + rel) of k * dt_min, k a power of two."""
    if not (dt_new > 0) or not math.isfinite(dt_new):
        return False
    q = math.log2(dt_new / DT_MIN)
    return abs(q - round(q)) <= rel / math.log(2)


def _check_corrections(st0, st1, idx, T, a1, j1, tsym=False):
    """Each active particle's corrected x, v and new step (st1) against the
    oracle's chain from st0 and the end-point force (a1, j1): the Hermite
    corrector (prediction, Hermite derivatives, correction) or, with tsym, the
    time-symmetric one; returns the worst error / bound ratios and the number of
    step decisions taken at a boundary."""
    worst_x = worst_v = 0.0
    flips = 0
    for k, i in enumerate(idx):
        x0, v0, a0, j0 = st0["x"][i], st0["v"][i], st0["a"][i], st0["j"][i]
        dt = (T - st0["tau"][i]) * DT_MIN
        xo, vo = oracle.predict_one(x0, v0, a0, j0, dt)
        a2, a3 = oracle.hermite_derivs(a0, j0, a1[k], j1[k], dt)
        da = np.abs(a0 - a1[k])
        S2 = 6 * da + dt * (4 * np.abs(j0) + 2 * np.abs(j1[k]))
        S3 = 12 * da + 6 * dt * (np.abs(j0) + np.abs(j1[k]))
        if tsym:
            x1, v1 = oracle.correct4s_one(x0, v0, a0, j0, a1[k], j1[k], dt)
            h = dt / 2
            # the FP32 velocity term h (a1 + a0) - h^2/3 (j1 - j0) and the double-single
            # sums; the position adds h (v1 + v0) (exact product of the hi part) and the
            # FP32 term h^2/3 (a1 - a0), and inherits h times the velocity's error
            bv = 4 * U48 * np.abs(v1) + 4 * U24 * (h * (np.abs(a1[k]) + np.abs(a0))
                                                   + h * h * (np.abs(j1[k]) + np.abs(j0)) / 3)
            bx = 4 * U48 * (np.abs(x1) + 2 * h * (np.abs(v0) + np.abs(v1))) \
                + 4 * U24 * h * h * (np.abs(a1[k]) + np.abs(a0)) / 3 + h * bv
        else:
            x1, v1 = oracle.correct_one(xo, vo, a2, a3, dt)
            bx, _ = _pred_bounds(x0, v0, a0, j0, vo, dt)
            bx = bx + 8 * U24 * (S2 / 24 + S3 / 120) * dt * dt + 4 * U48 * np.abs(x1)
            bv = 4 * U48 * np.abs(v0) + 4 * U24 * (np.abs(a0) * dt + np.abs(j0) * dt * dt / 2) \
                + 8 * U24 * (S2 / 6 + S3 / 24) * dt + 2.0 ** -44 * np.abs(v1)
        ex, ev = np.abs(st1["x"][i] - x1), np.abs(st1["v"][i] - v1)
        assert (ex <= bx).all(), (T, i, ex, bx)
        assert (ev <= bv).all(), (T, i, ev, bv)
        worst_x = max(worst_x, float((ex / bx).max()))
        worst_v = max(worst_v, float((ev / bv).max()))
        # new block step
        a2e = a2 + dt * a3
        dt_new = oracle.aarseth_dt(a1[k], j1[k], a2e, a3, ETA)
        want = oracle.quantise(dt_new, int(st0["dtau"][i]), int(T), DT_MIN, DTAU_MAX)
        if st1["dtau"][i] != want:
            # relative error of the estimate from the rounding of a2, a3 and the norms
            e2 = 4 * U24 * np.linalg.norm(S2) / dt ** 2
            e3 = 4 * U24 * np.linalg.norm(S3) / dt ** 3
            na1, nj1 = np.linalg.norm(a1[k]), np.linalg.norm(j1[k])
            na2, na3 = np.linalg.norm(a2e), np.linalg.norm(a3)
            num = na1 * na2 + nj1 ** 2
            den = nj1 * na3 + na2 ** 2
            r = 0.5 * ((na1 * (e2 + dt * e3)) / num + (nj1 * e3 + 2 * na2 * (e2 + dt * e3)) / den) + 16 * U24
            assert _near_boundary(dt_new, 4 * r), (T, i, st1["dtau"][i], want, dt_new, r)
            flips += 1
    return worst_x, worst_v, flips


@pytest.mark.parametrize("corrector", ["hermite", "timesym"])
def test_mixed_corrector_and_step_match_oracle_elementwise(corrector):
    """Sixty consecutive block steps of an integrated N = 2048 system: each
    active particle's corrected position and velocity against the oracle's
    prediction, Hermite derivatives and correction (or its time-symmetric
    corrector) from the same state and the same end-point force (the GPU's own,
    read through the force hook), and its new block step against the oracle's
    Aarseth step and quantisation."""
    n = 2048
    m, x, v = inputs.plummer(n, seed=33)
    checked = flips = 0
    worst_x = worst_v = 0.0
    tsym = corrector == "timesym"
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", corrector=corrector) as g:
        g.evolve(0.125)
        for _ in range(60):
            st0 = g.state()
            idx, T = g.active()
            a1, j1 = g.force(T, idx)
            g.replay_step(T, idx)
            st1 = g.state()
            others = np.setdiff1d(np.arange(n), idx)
            for k in ("x", "v", "a", "j", "tau", "dtau"):
                assert np.array_equal(st1[k][others], st0[k][others]), k
            # the corrector keeps exactly the force the hook returns
            assert np.array_equal(st1["a"][idx], a1) and np.array_equal(st1["j"][idx], j1)
            assert (st1["tau"][idx] == T).all()
            wx, wv, fl = _check_corrections(st0, st1, idx, T, a1, j1, tsym)
            worst_x, worst_v = max(worst_x, wx), max(worst_v, wv)
            flips += fl
            checked += idx.size
    print(corrector + " corrector: %d corrections, worst |dx|/bound %.3f |dv|/bound %.3f, %d step decisions at a boundary"
          % (checked, worst_x, worst_v, flips))
    assert checked > 500
    assert flips <= 0.01 * checked


@pytest.mark.parametrize("corrector", ["hermite", "timesym"])
def test_cluster_step_force_and_correction_match_oracle(corrector):
    """Block steps taken inside the small-step cluster (the kernel gd_evolve uses
    for steps with few active particles), one at a time: the end-point force the
    cluster computed (kept as the particles' new a and jerk) against the oracle's
    force on its own FP64 prediction of every particle, and the correction and
    new step against the oracle's chain from that force.  The cluster sums in
    FP32 without compensation: a lane adds up to ceil(P/32) terms of the CTA's P
    particles, then 5 shuffle levels, up to 4 levels of j-segments and 4 levels
    over the 16 CTAs, each addition rounding once, on top of the about 8 units of
    2^-24 a term carries."""
    n = 4096
    m, x, v = inputs.plummer(n, seed=35)
    rel_a, rel_j = [], []
    worst = [0.0, 0.0]
    flips = taken = 0
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", corrector=corrector) as g:
        csize, per_cta, ns = g.cluster_info()
        assert csize in (8, 16)
        bound = (8 + math.ceil(per_cta / 32) + 13) * U24
        g.evolve(0.125)
        for _ in range(120):
            st0 = g.state()
            idx, T = g.active()
            if idx.size > ns:
                t, k = g.step_block_small()
                assert (t, k) == (0.0, 0)  # too large for the cluster: left untaken
                g.step_block()
                continue
            t, k = g.step_block_small()
            assert k == idx.size and t == T * DT_MIN
            st1 = g.state()
            a1, j1 = st1["a"][idx], st1["j"][idx]
            xp, vp = oracle.predict_all(st0["x"], st0["v"], st0["a"], st0["j"], (T - st0["tau"]) * DT_MIN)
            a_or, j_or = oracle.force(m, xp, vp, EPS, idx)
            an, jn = oracle.force_absnorm(m, xp, vp, EPS, idx)
            assert (np.abs(a1 - a_or).max(axis=1) <= bound * an).all()
            assert (np.abs(j1 - j_or).max(axis=1) <= bound * jn).all()
            rel_a.extend((np.linalg.norm(a1 - a_or, axis=1) / np.linalg.norm(a_or, axis=1)).tolist())
            rel_j.extend((np.linalg.norm(j1 - j_or, axis=1) / np.linalg.norm(j_or, axis=1)).tolist())
            others = np.setdiff1d(np.arange(n), idx)
            for key in ("x", "v", "a", "j", "tau", "dtau"):
                assert np.array_equal(st1[key][others], st0[key][others]), key
            wx, wv, fl = _check_corrections(st0, st1, idx, T, a1, j1, corrector == "timesym")
            worst = [max(worst[0], wx), max(worst[1], wv)]
            flips += fl
            taken += idx.size
    ra, rj = np.array(rel_a), np.array(rel_j)
    print(corrector + " cluster steps: %d corrections; rel |da|/|a| median %.2e p99 %.2e max %.2e, |dj|/|j| median %.2e p99 %.2e "
          "max %.2e; worst |dx|/bound %.3f |dv|/bound %.3f; %d decisions at a boundary"
          % (taken, np.median(ra), np.percentile(ra, 99), ra.max(), np.median(rj), np.percentile(rj, 99), rj.max(),
             worst[0], worst[1], flips))
    assert taken > 300
    assert flips <= 0.01 * taken
    assert np.median(ra) <= 1e-6 and np.median(rj) <= 1e-6
