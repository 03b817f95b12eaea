"""Pins of the time-symmetric Hermite schemes in the oracle (hermite6_oracle.c,
order 4 and the P(EC)^n passes of either order) against what the mathematics
fixes: the fourth-order time-symmetric corrector against GraviDy's standard
corrector (an independent routine) through the Hermite quadrature's error term,
exactness on polynomial motion, fourth-order convergence, time reversibility of
the iterated map and the absence of a secular energy drift on a Kepler orbit.
"""
import math

import numpy as np
import pytest

from kepler import kepler_at, kepler_ic

DT_MIN = 2.0 ** -22


def _poly(coef, t, d):
    """d-th derivative at t of sum_k coef[k] t^k / k!  (coef: [K][3])."""
    out = np.zeros(3)
    for k in range(d, len(coef)):
        out += coef[k] * t ** (k - d) / math.factorial(k - d)
    return out


def test_time_symmetric_corrector_against_the_standard_one(oracle_mod):
    """Both correctors integrate the same cubic interpolant of (a, jerk): the
    velocities agree, and the time-symmetric position is the Hermite quadrature
    of that quartic velocity, whose error term gives
        x_sym = x_std - a''' dt^5 / 720
    with a''' the cubic's third derivative (GraviDy's standard corrector:
    prediction plus the a'' and a''' terms)."""
    rng = np.random.default_rng(11)
    for dt in (0.3, 0.1, 0.03):
        x0, v0, a0, j0, a1, j1 = (rng.normal(size=3) for _ in range(6))
        xs, vs = oracle_mod.correct4s_one(x0, v0, a0, j0, a1, j1, dt)
        xp, vp = oracle_mod.predict_one(x0, v0, a0, j0, dt)
        a2, a3 = oracle_mod.hermite_derivs(a0, j0, a1, j1, dt)
        xstd, vstd = oracle_mod.correct_one(xp, vp, a2, a3, dt)
        scale = np.abs(a3).max() * dt ** 5 / 720
        assert np.allclose(vs, vstd, rtol=1e-12, atol=1e-12 * np.abs(vstd).max())
        assert np.allclose(xs - xstd, -a3 * dt ** 5 / 720, rtol=1e-6, atol=1e-6 * scale)


def test_time_symmetric_corrector_exact_for_low_degree_motion(oracle_mod):
    """x(t) of degree 4: both formulas are exact.  Degree 5 (a cubic
    acceleration): the velocity is still exact, the position is off by the
    quadrature's error term.  Degree 6: neither is exact."""
    rng = np.random.default_rng(12)
    dt = 0.37
    for deg, v_exact, x_exact in ((4, True, True), (5, True, False), (6, False, False)):
        coef = rng.normal(size=(deg + 1, 3))
        x0, v0, a0, j0 = (_poly(coef, 0.0, d) for d in range(4))
        a1, j1 = (_poly(coef, dt, d) for d in (2, 3))
        x1, v1 = oracle_mod.correct4s_one(x0, v0, a0, j0, a1, j1, dt)
        dx = np.abs(x1 - _poly(coef, dt, 0)).max()
        dv = np.abs(v1 - _poly(coef, dt, 1)).max()
        assert (dv < 1e-13) == v_exact and (dx < 1e-13) == x_exact, (deg, dx, dv)


@pytest.mark.parametrize("order", [4, 6])
def test_corrector_is_time_symmetric(order, oracle_mod):
    """Correcting back from the end state with the ends swapped and -dt returns
    the start state (the defining property of the time-symmetric formulas)."""
    rng = np.random.default_rng(13)
    dt = 0.21
    x0, v0, a0, j0, s0, a1, j1, s1 = (rng.normal(size=3) for _ in range(8))
    if order == 4:
        x1, v1 = oracle_mod.correct4s_one(x0, v0, a0, j0, a1, j1, dt)
        xb, vb = oracle_mod.correct4s_one(x1, v1, a1, j1, a0, j0, -dt)
    else:
        x1, v1 = oracle_mod.correct6_one(x0, v0, a0, j0, s0, a1, j1, s1, dt)
        xb, vb = oracle_mod.correct6_one(x1, v1, a1, j1, s1, a0, j0, s0, -dt)
    assert np.allclose(xb, x0, rtol=0, atol=1e-14) and np.allclose(vb, v0, rtol=0, atol=1e-14)


def test_order4_time_symmetric_converges_at_fourth_order(oracle_mod):
    """Shared fixed steps on the e = 0.5 Kepler orbit, one and two passes:
    energy and position errors fall as dt^4."""
    def errs(dtau, n_iter, t_end=6.0):
        m, x, v = kepler_ic(0.5)
        sim = oracle_mod.Sim6(m, x, v, 0.0, 0.2, fixed_dtau=dtau, order=4, n_iter=n_iter)
        K0, U0 = sim.energy()
        sim.evolve(t_end)
        K, U = sim.energy()
        st = sim.state()
        r_ex, _ = kepler_at(t_end)
        return abs((K + U) / (K0 + U0) - 1), np.abs(st["x"][1] - st["x"][0] - r_ex).max()

    for n_iter in (1, 2):
        e = [errs(2 ** k, n_iter) for k in (15, 14, 13)]
        de = [math.log2(e[i][0] / e[i + 1][0]) for i in range(2)]
        dx = [math.log2(e[i][1] / e[i + 1][1]) for i in range(2)]
        print("H4 time-symmetric n_iter %d: slopes energy %s position %s" % (n_iter, de, dx))
        assert all(3.7 < s < 4.3 for s in de + dx), (de, dx)


def _round_trip(oracle_mod, order, n_iter, dtau=2 ** 14, steps=1536):
    """Forward `steps` shared steps, velocities reversed, forward again: the
    distance from the initial state (an exactly reversible map returns)."""
    m, x, v = kepler_ic(0.5)
    fwd = oracle_mod.Sim6(m, x, v, 0.0, 0.2, fixed_dtau=dtau, order=order, n_iter=n_iter)
    for _ in range(steps):
        fwd.step()
    st = fwd.state()
    back = oracle_mod.Sim6(m, st["x"], -st["v"], 0.0, 0.2, fixed_dtau=dtau, order=order, n_iter=n_iter)
    for _ in range(steps):
        back.step()
    sb = back.state()
    return max(np.abs(sb["x"] - x).max(), np.abs(sb["v"] + v).max())


@pytest.mark.parametrize("order", [4, 6])
def test_iterated_passes_make_the_map_reversible(order, oracle_mod):
    """About one orbit of shared steps dt = 2^-8 and back: two passes return to
    round-off; one pass (the corrector applied once to a predicted force) does
    not."""
    one = _round_trip(oracle_mod, order, 1)
    two = _round_trip(oracle_mod, order, 2)
    three = _round_trip(oracle_mod, order, 3)
    print("order %d round trip: one pass %.2e, two %.2e, three %.2e" % (order, one, two, three))
    assert two < 1e-13 and three < 1e-13
    assert one > 30 * max(two, three)


@pytest.mark.parametrize("order,dtau,bound", [(4, 2 ** 14, 1e-3), (6, 2 ** 15, 2e-2)])
def test_no_secular_energy_drift_with_two_passes(order, dtau, bound, oracle_mod):
    """Eight orbits of shared steps: the mean energy error of each orbit stays
    put with two passes, and drifts linearly with one."""
    nper = int(round(2 * math.pi / (dtau * DT_MIN)))

    def orbit_means(n_iter, norb=8):
        m, x, v = kepler_ic(0.5)
        sim = oracle_mod.Sim6(m, x, v, 0.0, 0.2, fixed_dtau=dtau, order=order, n_iter=n_iter)
        K0, U0 = sim.energy()
        err = []
        for _ in range(norb * nper):
            sim.step()
            K, U = sim.energy()
            err.append((K + U) / (K0 + U0) - 1)
        return np.array(err).reshape(norb, nper).mean(axis=1)

    for n_iter in (1, 2):
        means = orbit_means(n_iter)
        slope = np.polyfit(np.arange(len(means)), means, 1)[0]
        rel = abs(slope) * (len(means) - 1) / abs(means.mean())
        print("order %d n_iter %d: orbit means %s, drift over the run %.2e of the mean"
              % (order, n_iter, " ".join("%.3e" % q for q in means), rel))
        if n_iter == 1:
            assert rel > 0.1
        else:
            assert rel < bound


def test_block_steps_free_run_plummer(oracle_mod):
    """Block steps on a Plummer sphere to t = 1/4: the time-symmetric
    fourth-order scheme (one pass) takes about as many block steps as GraviDy's
    at the same eta and keeps an energy error of the same size, and so does a
    second pass, which doubles the evaluations: the interaction counter is the
    initial N^2 plus n_iter N per particle step."""
    from paper_1702_00440_gb300 import inputs
    m, x, v = inputs.plummer(256, seed=9)
    std = oracle_mod.Sim(m, x, v, 1e-4, 0.01)
    E = sum(std.energy())
    std.evolve(0.25)
    d_std = abs(sum(std.energy()) / E - 1)
    res = {}
    for n_iter in (1, 2):
        ts = oracle_mod.Sim6(m, x, v, 1e-4, 0.01, eta_init=0.01, order=4, n_iter=n_iter)
        ts.evolve(0.25)
        res[n_iter] = (abs(sum(ts.energy()) / E - 1), ts.stats())
    nb = std.stats()["nblock"]
    print("standard: dE %.2e blocks %d; time-symmetric 1 pass: dE %.2e blocks %d; 2 passes: dE %.2e blocks %d"
          % (d_std, nb, res[1][0], res[1][1]["nblock"], res[2][0], res[2][1]["nblock"]))
    for n_iter in (1, 2):
        st = res[n_iter][1]
        assert abs(st["nblock"] - nb) < 0.05 * nb
        assert res[n_iter][0] < 2 * d_std
        assert st["interactions"] == 256.0 * 256 + n_iter * 256.0 * st["nsteps"]
