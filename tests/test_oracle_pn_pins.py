"""Pins of the oracle's post-Newtonian pair terms (Sec. 5: corrections for an
eps = 0 binary; the 1PN and 2.5PN two-body accelerations in harmonic
coordinates) against facts they must reproduce, not against a retyped formula:

- the jerk is the time derivative of the acceleration along the motion
  (Richardson-extrapolated central differences of the acceleration itself);
- 1PN: an eccentric binary's periastron advances by 6 pi M / (c^2 a (1 - e^2))
  per orbit (Einstein; e.g. Robertson 1938, Damour & Deruelle 1985);
- 2.5PN: the orbit-averaged decay of the semi-major axis and eccentricity
  follows Peters (1964): da/dt = -64/5 eta M^3 / (c^5 a^3 (1 - e^2)^(7/2))
  (1 + 73/24 e^2 + 37/96 e^4), de/dt = -304/15 eta M^3 e / (c^5 a^4
  (1 - e^2)^(5/2)) (1 + 121/304 e^2);
- the pair's terms conserve its momentum (shares m_q/M and -m_p/M).
"""
import numpy as np
import pytest

import oracle

M1, M2 = 0.6, 0.4
M = M1 + M2
ETA = M1 * M2 / M ** 2
DT_MIN = 2.0 ** -22


@pytest.fixture(scope="module", autouse=True)
def _built(oracle_mod):
    return oracle_mod


def _binary(a, e):
    """The pair at periastron, centre of mass at rest at the origin."""
    r = np.array([a * (1 - e), 0.0, 0.0])
    v = np.array([0.0, np.sqrt(M * (1 + e) / (a * (1 - e))), 0.0])
    x = np.stack([M2 / M * r, -M1 / M * r])
    vv = np.stack([M2 / M * v, -M1 / M * v])
    return np.array([M1, M2]), x, vv


@pytest.mark.parametrize("terms", [oracle.PN_1, oracle.PN_25, oracle.PN_1 | oracle.PN_25])
def test_pn_jerk_is_the_derivative_of_the_acceleration(terms):
    rng = np.random.default_rng(terms)
    for _ in range(5):
        r0 = rng.normal(size=3)
        v0 = rng.normal(size=3) * 0.7
        ar = rng.normal(size=3) * 0.5
        c = 7.0

        def acc(t):
            return oracle.pn_accel(M1, M2, r0 + v0 * t + 0.5 * ar * t * t, v0 + ar * t, c, terms)

        d = lambda h: (acc(h) - acc(-h)) / (2 * h)
        h = 1e-3
        rich = (4 * d(h / 2) - d(h)) / 3  # error O(h^4)
        j = oracle.pn_jerk(M1, M2, r0, v0, ar, c, terms)
        assert np.abs(j - rich).max() <= 1e-9 * np.abs(j).max()


def _orbit_track(terms, c, a, e, orbits, fixed_dtau=1 << 12):
    m, x, v = _binary(a, e)
    sim = oracle.Sim(m, x, v, 0.0, 0.01, fixed_dtau=fixed_dtau, dt_max=0.125)
    sim.set_pn(0, 1, c, terms)
    period = 2 * np.pi * np.sqrt(a ** 3 / M)
    t_end = orbits * period
    ts, rs, vs, ps = [], [], [], []
    while True:
        tick, _ = sim.step()
        st = sim.state()
        ts.append(tick * DT_MIN)
        rs.append(st["x"][0] - st["x"][1])
        vs.append(st["v"][0] - st["v"][1])
        ps.append(M1 * st["v"][0] + M2 * st["v"][1])
        if ts[-1] >= t_end:
            break
    return np.array(ts), np.array(rs), np.array(vs), np.array(ps)


def test_1pn_periastron_advance_matches_the_relativistic_formula():
    a, e = 1.0, 0.5
    res = {}
    for c in (30.0, 100.0):
        res[c] = _advance(c, a, e)
    # the relative departure from the leading-order formula is of order M / (c^2 a):
    # about 1e-3 at c = 30, ten times smaller at c = 100
    assert abs(res[30.0] - 1) < 0.01
    assert abs(res[100.0] - 1) < 0.002
    assert abs(res[100.0] - 1) < 0.2 * abs(res[30.0] - 1)


def _advance(c, a, e):
    ts, rs, vs, ps = _orbit_track(oracle.PN_1, c, a, e, 6)
    rr = np.linalg.norm(rs, axis=1)
    ang = np.unwrap(np.arctan2(rs[:, 1], rs[:, 0]))
    # periastron passages: local minima of |r|, angle refined by a parabola in time
    peri = []
    for k in range(1, rr.size - 1):
        if rr[k] < rr[k - 1] and rr[k] <= rr[k + 1]:
            y0, y1, y2 = rr[k - 1], rr[k], rr[k + 1]
            s = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)  # offset of the minimum in steps
            a0, a1, a2 = ang[k - 1], ang[k], ang[k + 1]
            peri.append(a1 + s * 0.5 * (a2 - a0) + s * s * 0.5 * (a2 - 2 * a1 + a0))
    peri = np.array(peri)
    assert peri.size >= 5
    adv = np.diff(peri) - 2 * np.pi
    want = 6 * np.pi * M / (c * c * a * (1 - e * e))
    print("1PN periastron advance per orbit at c = %g: measured %.6e (spread %.1e), formula %.6e"
          % (c, adv.mean(), adv.std(), want))
    # the pair's momentum is conserved (its centre of mass stays at rest)
    assert np.abs(ps).max() < 1e-13
    return adv.mean() / want


def _elements(rs, vs):
    rr = np.linalg.norm(rs, axis=1)
    v2 = np.einsum("ij,ij->i", vs, vs)
    E = 0.5 * v2 - M / rr
    a = -M / (2 * E)
    L = np.cross(rs, vs)
    lrl = np.cross(vs, L) - M * rs / rr[:, None]
    e = np.linalg.norm(lrl, axis=1) / M
    return a, e


def test_25pn_orbit_decay_follows_peters():
    a0, e0, c = 1.0, 0.3, 10.0
    orbits = 6
    ts, rs, vs, ps = _orbit_track(oracle.PN_25, c, a0, e0, orbits)
    a, e = _elements(rs, vs)
    period = 2 * np.pi * np.sqrt(a0 ** 3 / M)
    # orbit averages over whole periods, then the mean rate between the first and last
    k = np.floor(ts / period).astype(int)
    sel = [k == q for q in range(orbits)]
    am = np.array([a[s].mean() for s in sel])
    em = np.array([e[s].mean() for s in sel])
    tm = np.array([ts[s].mean() for s in sel])
    dadt = np.polyfit(tm, am, 1)[0]
    dedt = np.polyfit(tm, em, 1)[0]
    aa, ee = am.mean(), em.mean()
    pa = -64 / 5 * ETA * M ** 3 / (c ** 5 * aa ** 3 * (1 - ee ** 2) ** 3.5) * (1 + 73 / 24 * ee ** 2 + 37 / 96 * ee ** 4)
    pe = -304 / 15 * ETA * M ** 3 * ee / (c ** 5 * aa ** 4 * (1 - ee ** 2) ** 2.5) * (1 + 121 / 304 * ee ** 2)
    print("2.5PN decay: da/dt %.5e (Peters %.5e), de/dt %.5e (Peters %.5e)" % (dadt, pa, dedt, pe))
    # leading-order radiation reaction on a Newtonian orbit: the measured rates agree
    # to a few parts in 1e5; a wrong coefficient of either 2.5PN term moves them by
    # tens of percent
    assert abs(dadt / pa - 1) < 1e-3
    assert abs(dedt / pe - 1) < 1e-3
    assert np.abs(ps).max() < 1e-13


def test_pn_pair_rejects_bad_arguments():
    m, x, v = _binary(1.0, 0.1)
    sim = oracle.Sim(m, x, v, 0.0, 0.01)
    with pytest.raises(ValueError):
        sim.set_pn(0, 0, 10.0)
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, -1.0)
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, 10.0, terms=2)  # 2PN is not built
    sim.set_pn(0, 1, 10.0)
    sim.step()
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, 10.0)  # after the first step
