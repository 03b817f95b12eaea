"""Pins of the FP64 oracle against values the paper and the mathematics fix.

Each test checks the oracle against something other than its own formula:
hand-derived values, closed forms (Kepler orbits, circular-orbit derivatives),
exactness on polynomial motion, conservation laws and symmetries, finite
differences, the convergence order, and the paper's printed example run.
"""
import json
import math
import os

import numpy as np
import pytest

from kepler import kepler_at as _kepler_at
from kepler import kepler_ic as _kepler_ic
from paper_1702_00440_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DT_MIN = 2.0 ** -22


def _ev(expr):
    return eval(expr, {"sqrt": math.sqrt, "__builtins__": {}})


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- force/jerk

def test_n3_hand_forces_and_energy(oracle_mod):
    g = _golden("n3_hand.json")
    m, x, v = np.array(g["m"]), np.array(g["x"], float), np.array(g["v"], float)
    for case in g["cases"]:
        acc, jrk = oracle_mod.force(m, x, v, case["eps"])
        want_a = np.array([[_ev(e) for e in row] for row in case["acc"]])
        want_j = np.array([[_ev(e) for e in row] for row in case["jerk"]])
        np.testing.assert_allclose(acc, want_a, rtol=0, atol=1e-15)
        np.testing.assert_allclose(jrk, want_j, rtol=0, atol=1e-15)
        K, U = oracle_mod.energy(m, x, v, case["eps"])
        assert K == pytest.approx(_ev(case["K"]), abs=1e-15)
        assert U == pytest.approx(_ev(case["U"]), abs=1e-14)


def _rotation(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q


def test_rotation_permutation_galilean_covariance(oracle_mod):
    """a and jerk rotate with the system, follow a relabelling of the
    particles, and are unchanged by a uniform translation or boost."""
    m, x, v = inputs.plummer(64, seed=3)
    eps = 0.01
    a, j = oracle_mod.force(m, x, v, eps)
    R = _rotation(5)
    ar, jr = oracle_mod.force(m, x @ R.T, v @ R.T, eps)
    np.testing.assert_allclose(ar, a @ R.T, rtol=0, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(jr, j @ R.T, rtol=0, atol=1e-12 * np.abs(j).max())
    p = np.random.default_rng(7).permutation(64)
    ap, jp = oracle_mod.force(m[p], x[p], v[p], eps)
    np.testing.assert_allclose(ap, a[p], rtol=1e-13, atol=1e-13 * np.abs(a).max())
    np.testing.assert_allclose(jp, j[p], rtol=1e-13, atol=1e-13 * np.abs(j).max())
    at, jt = oracle_mod.force(m, x + np.array([0.3, -0.2, 0.1]), v + np.array([1.0, 2.0, -0.5]), eps)
    np.testing.assert_allclose(at, a, rtol=0, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(jt, j, rtol=0, atol=1e-11 * np.abs(j).max())


def test_pairwise_antisymmetry_and_zero_torque(oracle_mod):
    """Newton's third law: sum m a = 0, sum m jerk = 0, sum m x cross a = 0."""
    m, x, v = inputs.plummer(512, seed=2, masses=inputs.power_law_masses(512, seed=2))
    a, j = oracle_mod.force(m, x, v, 1e-4)
    an, jn = oracle_mod.force_absnorm(m, x, v, 1e-4)
    sa = (m * an).sum()
    sj = (m * jn).sum()
    assert np.abs((m[:, None] * a).sum(0)).max() < 1e-14 * sa
    assert np.abs((m[:, None] * j).sum(0)).max() < 1e-14 * sj
    torque = (m[:, None] * np.cross(x, a)).sum(0)
    assert np.abs(torque).max() < 1e-14 * (m * an * np.linalg.norm(x, axis=1)).sum()


def test_jerk_is_time_derivative_of_acceleration(oracle_mod):
    """Central difference of a along straight-line motion x + v t matches the
    jerk to O(h^2)."""
    m, x, v = inputs.plummer(48, seed=4)
    eps = 0.05
    _, j = oracle_mod.force(m, x, v, eps)
    errs = []
    for h in (1e-3, 5e-4):
        ap, _ = oracle_mod.force(m, x + h * v, v, eps)
        am, _ = oracle_mod.force(m, x - h * v, v, eps)
        fd = (ap - am) / (2 * h)
        errs.append(np.abs(fd - j).max() / np.abs(j).max())
    assert errs[0] < 1e-4
    assert errs[1] < errs[0] / 3.0  # second-order convergence of the difference


def test_potential_is_consistent_with_force(oracle_mod):
    """dU/dt along straight-line motion equals - sum_i m_i v_i . a_i (the force
    is minus the gradient of the softened potential)."""
    m, x, v = inputs.plummer(48, seed=6)
    eps = 0.05
    a, _ = oracle_mod.force(m, x, v, eps)
    h = 1e-5
    _, up = oracle_mod.energy(m, x + h * v, v, eps)
    _, um = oracle_mod.energy(m, x - h * v, v, eps)
    dudt = (up - um) / (2 * h)
    want = -(m[:, None] * v * a).sum()
    assert dudt == pytest.approx(want, rel=1e-6)


def test_absnorm_equals_magnitude_for_a_single_term(oracle_mod):
    m = np.array([1.0, 2.0])
    x = np.array([[0.0, 0, 0], [0.3, -0.4, 0.0]])
    v = np.array([[0.0, 0, 0], [0.0, 0.0, 0.7]])  # r perpendicular to v
    a, j = oracle_mod.force(m, x, v, 0.1)
    an, jn = oracle_mod.force_absnorm(m, x, v, 0.1)
    np.testing.assert_allclose(an, np.linalg.norm(a, axis=1), rtol=1e-15)
    np.testing.assert_allclose(jn, np.linalg.norm(j, axis=1), rtol=1e-15)


# ---------------------------------------------------------------- active list

def test_active_list_is_the_definition(oracle_mod):
    rng = np.random.default_rng(11)
    for n in (1, 2, 31, 32, 33, 1000):
        for _ in range(5):
            t = rng.integers(0, 4, size=n).astype(np.int64) * 8 + 8
            idx, tn = oracle_mod.active(t)
            assert tn == t.min()
            assert idx.tolist() == [i for i in range(n) if t[i] == tn]
    t = np.full(77, 5, np.int64)
    idx, tn = oracle_mod.active(t)
    assert idx.tolist() == list(range(77)) and tn == 5
    t[-1] = 4
    idx, tn = oracle_mod.active(t)
    assert idx.tolist() == [76] and tn == 4


# ------------------------------------------------- predictor / corrector / dt

def _poly_motion(seed):
    rng = np.random.default_rng(seed)
    X0, V0, A0, A1, A2, A3 = (rng.normal(size=3) for _ in range(6))
    return X0, V0, A0, A1, A2, A3


def test_predictor_reproduces_cubic_motion(oracle_mod):
    X0, V0, A0, A1, _, _ = _poly_motion(1)
    dt = 0.37
    xp, vp = oracle_mod.predict_one(X0, V0, A0, A1, dt)
    for c in range(3):
        px = np.polynomial.Polynomial([X0[c], V0[c], A0[c] / 2, A1[c] / 6])
        assert xp[c] == pytest.approx(px(dt), abs=1e-14)
        assert vp[c] == pytest.approx(px.deriv()(dt), abs=1e-14)


def test_hermite_interpolation_is_exact_for_cubic_acceleration(oracle_mod):
    """If a(t) is a cubic, the end-point values fix its 2nd and 3rd derivative
    at the start exactly."""
    _, _, A0, A1, A2, A3 = _poly_motion(2)
    for dt in (0.5, 2.0 ** -7):
        pa = [np.polynomial.Polynomial([A0[c], A1[c], A2[c] / 2, A3[c] / 6]) for c in range(3)]
        a0 = np.array([p(0.0) for p in pa])
        j0 = np.array([p.deriv()(0.0) for p in pa])
        a1 = np.array([p(dt) for p in pa])
        j1 = np.array([p.deriv()(dt) for p in pa])
        a2, a3 = oracle_mod.hermite_derivs(a0, j0, a1, j1, dt)
        scale = 1e-13 / dt ** 3
        np.testing.assert_allclose(a2, A2, rtol=0, atol=scale * dt)
        np.testing.assert_allclose(a3, A3, rtol=0, atol=scale)


def test_corrector_is_exact_for_quintic_motion(oracle_mod):
    """Predict with (x, v, a, jerk), interpolate a2, a3, correct: for motion
    whose acceleration is a cubic in time the result is the exact quintic."""
    X0, V0, A0, A1, A2, A3 = _poly_motion(3)
    dt = 0.25
    px = [np.polynomial.Polynomial([X0[c], V0[c], A0[c] / 2, A1[c] / 6, A2[c] / 24, A3[c] / 120]) for c in range(3)]
    pv = [p.deriv() for p in px]
    pa = [p.deriv(2) for p in px]
    pj = [p.deriv(3) for p in px]
    a1 = np.array([p(dt) for p in pa])
    j1 = np.array([p(dt) for p in pj])
    xp, vp = oracle_mod.predict_one(X0, V0, A0, A1, dt)
    a2, a3 = oracle_mod.hermite_derivs(A0, A1, a1, j1, dt)
    x1, v1 = oracle_mod.correct_one(xp, vp, a2, a3, dt)
    np.testing.assert_allclose(x1, [p(dt) for p in px], rtol=0, atol=1e-14)
    np.testing.assert_allclose(v1, [p(dt) for p in pv], rtol=0, atol=1e-14)


def test_aarseth_step_on_circular_orbit(oracle_mod):
    """On a circular orbit of angular frequency w the derivatives have
    magnitudes w^2 r, w^3 r, w^4 r, w^5 r, so the criterion gives sqrt(eta)/w."""
    r, w, eta = 1.7, 0.8, 0.01
    th = 0.3
    c, s = math.cos(th), math.sin(th)
    a1 = -w ** 2 * r * np.array([c, s, 0])
    j1 = -w ** 3 * r * np.array([-s, c, 0])
    a2 = w ** 4 * r * np.array([c, s, 0])
    a3 = w ** 5 * r * np.array([-s, c, 0])
    assert oracle_mod.aarseth_dt(a1, j1, a2, a3, eta) == pytest.approx(math.sqrt(eta) / w, rel=1e-14)


def test_block_quantisation_rules(oracle_mod):
    q0 = oracle_mod.quantise_init
    dmax = 2 ** 19
    assert q0(0.1, DT_MIN, dmax) == 2 ** 18          # 2^-4 = 0.0625 <= 0.1 < 2^-3
    assert q0(0.125, DT_MIN, dmax) == dmax
    assert q0(5.0, DT_MIN, dmax) == dmax
    assert q0(float("inf"), DT_MIN, dmax) == dmax
    assert q0(float("nan"), DT_MIN, dmax) == dmax
    assert q0(1e-9, DT_MIN, dmax) == 1
    assert q0(2.0 ** -22, DT_MIN, dmax) == 1
    q = oracle_mod.quantise
    old = 2 ** 10
    assert q(old * DT_MIN * 0.3, old, 5 * old, DT_MIN, dmax) == 2 ** 8     # shrink freely
    assert q(old * DT_MIN * 0.999, old, 5 * old, DT_MIN, dmax) == 2 ** 9
    assert q(old * DT_MIN * 1.5, old, 4 * old, DT_MIN, dmax) == old        # no growth below 2x
    assert q(old * DT_MIN * 8.0, old, 4 * old, DT_MIN, dmax) == 2 * old    # grow x2 only
    assert q(old * DT_MIN * 8.0, old, 5 * old, DT_MIN, dmax) == old        # not commensurate
    assert q(dmax * DT_MIN * 4.0, dmax, 4 * dmax, DT_MIN, dmax) == dmax    # capped at dt_max
    assert q(1e-12, old, 5 * old, DT_MIN, dmax) == 1                       # clamped at dt_min
    assert q(float("nan"), old, 4 * old, DT_MIN, dmax) == 2 * old


# ---------------------------------------------------------------- integrator

def test_kepler_orbit_block_steps(oracle_mod):
    e = 0.5
    m, x, v = _kepler_ic(e)
    sim = oracle_mod.Sim(m, x, v, eps=0.0, eta=0.01)
    K0, U0 = sim.energy()
    assert K0 + U0 == pytest.approx(-0.5 * 0.5 / 2, rel=1e-14)   # -m1 m2 / (2a)
    t_end = 6.25                                                   # about one period (2 pi)
    sim.evolve(t_end)
    st = sim.state()
    assert (st["tau"] == int(t_end / DT_MIN)).all()
    r = st["x"][1] - st["x"][0]
    w = st["v"][1] - st["v"][0]
    r_ex, w_ex = _kepler_at(t_end, e)
    assert np.abs(r - r_ex).max() < 1e-4      # orbital phase error at eta = 0.01
    assert np.abs(w - w_ex).max() < 1e-4
    K, U = sim.energy()
    assert abs((K + U) / (K0 + U0) - 1) < 1e-6   # Sec. 3.2: ~1e-7 at eta = 0.01
    # eccentricity from the Laplace-Runge-Lenz vector
    L = np.cross(r, w)
    ecc = np.cross(w, L) - r / np.linalg.norm(r)
    assert np.linalg.norm(ecc) == pytest.approx(e, abs=1e-6)
    # momentum of the pair (both bodies always share the block step)
    assert np.abs((m[:, None] * st["v"]).sum(0)).max() < 1e-15


def _energy_error_fixed(oracle_mod, dtau, t_end=6.0):
    m, x, v = _kepler_ic(0.5)
    sim = oracle_mod.Sim(m, x, v, eps=0.0, eta=0.01, fixed_dtau=dtau)
    K0, U0 = sim.energy()
    sim.evolve(t_end)
    K, U = sim.energy()
    st = sim.state()
    r_ex, _ = _kepler_at(t_end)
    return abs((K + U) / (K0 + U0) - 1), np.abs(st["x"][1] - st["x"][0] - r_ex).max()


def test_fourth_order_convergence_shared_steps(oracle_mod):
    """Shared fixed steps: the energy and position errors fall as dt^4
    (Sec. 3.2: H4's error is O(dt^4) with a shared time step)."""
    errs = [_energy_error_fixed(oracle_mod, 2 ** k) for k in (16, 15, 14, 13)]
    de = [math.log2(errs[i][0] / errs[i + 1][0]) for i in range(3)]
    dx = [math.log2(errs[i][1] / errs[i + 1][1]) for i in range(3)]
    assert all(3.6 < s < 4.6 for s in de), de
    assert all(3.6 < s < 4.6 for s in dx), dx


def test_momentum_conserved_to_roundoff_with_shared_steps(oracle_mod):
    m, x, v = inputs.plummer(64, seed=9)
    sim = oracle_mod.Sim(m, x, v, eps=0.01, eta=0.01, fixed_dtau=2 ** 12)
    sim.evolve(0.25)
    st = sim.state()
    p = (m[:, None] * st["v"]).sum(0)
    assert np.abs(p).max() < 1e-15


def test_replay_reproduces_free_run_bit_for_bit(oracle_mod):
    m, x, v = inputs.plummer(128, seed=12)
    a = oracle_mod.Sim(m, x, v, eps=1e-4, eta=0.01)
    rec = [a.step() for _ in range(300)]
    b = oracle_mod.Sim(m, x, v, eps=1e-4, eta=0.01)
    for tick, idx in rec:
        b.replay(tick, idx)
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_block_schedule_invariants(oracle_mod):
    m, x, v = inputs.plummer(256, seed=1)
    sim = oracle_mod.Sim(m, x, v, eps=1e-4, eta=0.01)
    nsteps = 0
    seen_levels = set()
    dtau_max = int(0.125 / DT_MIN)
    while True:
        tick, idx = sim.step()
        nsteps += idx.size
        st = sim.state()
        assert (st["tau"] % st["dtau"] == 0).all()
        assert ((st["dtau"] & (st["dtau"] - 1)) == 0).all()    # powers of two
        assert st["dtau"].max() <= dtau_max
        assert (st["tau"][idx] == tick).all()
        seen_levels.update(np.unique(st["dtau"]).tolist())
        if tick == 2 * dtau_max:
            break
    assert (st["tau"] == 2 * dtau_max).all()                    # synchronised at 2 dt_max
    assert sim.stats()["nsteps"] == nsteps
    assert len(seen_levels) >= 3


@pytest.mark.slow
def test_paper_example_run_plausibility(oracle_mod):
    """N = 1024 Plummer to t = 1 with eta = 0.01: block and particle steps of
    the paper's Appendix A order of magnitude and Delta E / E small (Sec. 3.2)."""
    g = _golden("paper_appendix_a_run.json")
    m, x, v = inputs.plummer(g["n"], seed=1)
    sim = oracle_mod.Sim(m, x, v, eps=1e-4, eta=0.01)
    K0, U0 = sim.energy()
    sim.evolve(g["t_end"])
    K, U = sim.energy()
    s = sim.stats()
    assert g["block_steps"] / 1.5 < s["nblock"] < g["block_steps"] * 1.5
    assert g["particle_steps"] / 1.5 < s["nsteps"] < g["particle_steps"] * 1.5
    assert abs((K + U - K0 - U0) / (K0 + U0)) < 1e-5
