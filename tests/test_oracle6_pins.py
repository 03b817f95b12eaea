"""Pins of the sixth-order FP64 oracle (hermite6_oracle.c) against values the
mathematics fixes: the snap as the time derivative of the jerk, Newton's third
law, exactness of the predictor, interpolant and corrector on polynomial
motion, the step criterion on a circular orbit, a Kepler orbit against its
closed form, and sixth-order convergence under shared steps.
"""
import math

import numpy as np
import pytest

from kepler import kepler_at, kepler_ic
from paper_1702_00440_gb300 import inputs

DT_MIN = 2.0 ** -22


def test_force6_acc_jerk_equal_the_4th_order_oracle(oracle_mod):
    m, x, v = inputs.plummer(200, seed=3)
    a, j = oracle_mod.force(m, x, v, 1e-3)
    a6, j6, _ = oracle_mod.force6(m, x, v, a, 1e-3)
    assert np.abs(a6 - a).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(j6 - j).max() <= 1e-13 * np.abs(j).max()


def test_snap_is_the_time_derivative_of_the_jerk(oracle_mod):
    """Along x(t) = x + v t + b t^2 / 2 (every particle, b arbitrary) the jerk
    J(t) of the 4th-order oracle has dJ/dt(0) = snap(x, v, a = b); central
    differences converge to it as h^2."""
    rng = np.random.default_rng(5)
    m, x, v = inputs.plummer(40, seed=6)
    b = rng.normal(size=(40, 3))
    eps = 0.05
    _, _, snap = oracle_mod.force6(m, x, v, b, eps)

    def jerk(t):
        return oracle_mod.force(m, x + v * t + 0.5 * b * t * t, v + b * t, eps)[1]

    errs, fds = [], []
    for h in (2.5e-3, 1.25e-3, 6.25e-4):
        fd = (jerk(h) - jerk(-h)) / (2 * h)
        fds.append(fd)
        errs.append(np.abs(fd - snap).max() / np.abs(snap).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4   # O(h^2)
    # Richardson extrapolation removes the h^2 term: agreement to O(h^4)
    rich = (4 * fds[2] - fds[1]) / 3
    assert np.abs(rich - snap).max() / np.abs(snap).max() < 1e-6


def test_snap_antisymmetry(oracle_mod):
    m, x, v = inputs.plummer(300, seed=8, masses=inputs.power_law_masses(300, seed=8))
    a, _ = oracle_mod.force(m, x, v, 1e-4)
    _, _, s = oracle_mod.force6(m, x, v, a, 1e-4)
    tot = np.abs(m[:, None] * s).sum(0)
    assert np.all(np.abs((m[:, None] * s).sum(0)) <= 1e-12 * tot)


def _poly(coef, t, d):
    """d-th derivative at t of sum_k coef[k] t^k / k!  (coef: [K][3])."""
    out = np.zeros(3)
    for k in range(d, len(coef)):
        out += coef[k] * t ** (k - d) / math.factorial(k - d)
    return out


def test_predictor_exact_for_quintic_motion(oracle_mod):
    rng = np.random.default_rng(1)
    coef = rng.normal(size=(6, 3))
    dt = 0.37
    xp, vp, ap = oracle_mod.predict6_one(*(_poly(coef, 0, d) for d in range(6)), dt)
    assert np.allclose(xp, _poly(coef, dt, 0), rtol=1e-14, atol=1e-14)
    assert np.allclose(vp, _poly(coef, dt, 1), rtol=1e-14, atol=1e-14)
    assert np.allclose(ap, _poly(coef, dt, 2), rtol=1e-14, atol=1e-14)


def test_interpolant_derivatives_exact_for_quintic_acceleration(oracle_mod):
    """x(t) of degree 7 (a quintic acceleration): crackle, pop and the fifth
    derivative at the end of the step follow from a, jerk, snap at both ends."""
    rng = np.random.default_rng(2)
    coef = rng.normal(size=(8, 3))
    dt = 0.29
    end = [_poly(coef, dt, d) for d in (2, 3, 4)]
    beg = [_poly(coef, 0.0, d) for d in (2, 3, 4)]
    c, p, q = oracle_mod.derivs6(*beg, *end, dt)
    for got, d in ((c, 5), (p, 6), (q, 7)):
        want = _poly(coef, dt, d)
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(coef).max()), d


def test_corrector_exact_for_sextic_motion(oracle_mod):
    """x(t) of degree 6: the time-symmetric corrector's velocity (the integral of
    the quintic interpolant of the acceleration) and position (the same quadrature
    of the velocity, a quintic) are exact; a degree-7 term breaks the position."""
    rng = np.random.default_rng(3)
    dt = 0.41
    for deg, exact in ((6, True), (7, False)):
        coef = rng.normal(size=(deg + 1, 3))
        x0, v0, a0, j0, s0 = (_poly(coef, 0.0, d) for d in range(5))
        a1, j1, s1 = (_poly(coef, dt, d) for d in (2, 3, 4))
        x1, v1 = oracle_mod.correct6_one(x0, v0, a0, j0, s0, a1, j1, s1, dt)
        assert np.allclose(v1, _poly(coef, dt, 1), rtol=1e-13, atol=1e-13)
        dx = np.abs(x1 - _poly(coef, dt, 0)).max()
        assert (dx < 1e-13) == exact, (deg, dx)


def test_step_criterion_on_a_circular_orbit(oracle_mod):
    """Uniform circular motion with angular frequency w: |a^(k)| = w^(k+2) R, so
    the sixth-order criterion gives eta / w."""
    R, w, t = 1.7, 2.3, 0.4
    der = []
    for k in range(6):   # a, jerk, snap, crackle, pop, 5th derivative
        n = k + 2
        der.append(R * w ** n * np.array([math.cos(w * t + n * math.pi / 2), math.sin(w * t + n * math.pi / 2), 0.0]))
    assert oracle_mod.aarseth6_dt(*der, 0.3) == pytest.approx(0.3 / w, rel=1e-14)


def test_kepler_orbit_sixth_order_block_steps(oracle_mod):
    e, t_end = 0.5, 6.25
    m, x, v = kepler_ic(e)
    sim = oracle_mod.Sim6(m, x, v, eps=0.0, eta=0.2)
    K0, U0 = sim.energy()
    sim.evolve(t_end)
    st = sim.state()
    assert (st["tau"] == int(t_end / DT_MIN)).all()
    r = st["x"][1] - st["x"][0]
    w = st["v"][1] - st["v"][0]
    r_ex, w_ex = kepler_at(t_end, e)
    K, U = sim.energy()
    print("H6 kepler: |dr| %.2e |dE/E| %.2e blocks %d" % (np.abs(r - r_ex).max(), (K + U) / (K0 + U0) - 1,
                                                          sim.stats()["nblock"]))
    assert np.abs(r - r_ex).max() < 1e-5
    assert np.abs(w - w_ex).max() < 1e-5
    assert abs((K + U) / (K0 + U0) - 1) < 1e-7
    L = np.cross(r, w)
    ecc = np.cross(w, L) - r / np.linalg.norm(r)
    assert np.linalg.norm(ecc) == pytest.approx(e, abs=1e-7)


def test_sixth_order_convergence_shared_steps(oracle_mod):
    """Shared fixed steps on the e = 0.5 Kepler orbit: the energy and position
    errors fall as dt^6."""
    def errs(dtau, t_end=6.0):
        m, x, v = kepler_ic(0.5)
        sim = oracle_mod.Sim6(m, x, v, eps=0.0, eta=0.2, fixed_dtau=dtau)
        K0, U0 = sim.energy()
        sim.evolve(t_end)
        K, U = sim.energy()
        st = sim.state()
        r_ex, _ = kepler_at(t_end)
        return abs((K + U) / (K0 + U0) - 1), np.abs(st["x"][1] - st["x"][0] - r_ex).max()

    e = [errs(2 ** k) for k in (17, 16, 15)]
    de = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
    dx = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
    print("H6 slopes energy %s position %s" % (de, dx))
    assert all(5.3 < s < 6.8 for s in de), de
    assert all(5.3 < s < 6.8 for s in dx), dx


def test_sixth_order_beats_fourth_at_equal_cost(oracle_mod):
    """On the same Plummer sphere to t = 1/4, the sixth-order scheme at eta = 0.3
    takes fewer particle steps than the fourth-order one at eta = 0.01 and still
    has the smaller energy error."""
    m, x, v = inputs.plummer(128, seed=4)
    s4 = oracle_mod.Sim(m, x, v, 1e-3, 0.01)
    s6 = oracle_mod.Sim6(m, x, v, 1e-3, 0.3)
    E4, E6 = sum(s4.energy()), sum(s6.energy())
    s4.evolve(0.25)
    s6.evolve(0.25)
    d4 = abs((sum(s4.energy()) - E4) / E4)
    d6 = abs((sum(s6.energy()) - E6) / E6)
    n4, n6 = s4.stats()["nsteps"], s6.stats()["nsteps"]
    print("H4 eta 0.01: dE %.2e steps %d; H6 eta 0.3: dE %.2e steps %d" % (d4, n4, d6, n6))
    assert n6 < n4 and d6 < d4
