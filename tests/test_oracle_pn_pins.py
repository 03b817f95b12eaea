"""Pins of the oracle's post-Newtonian pair terms (Sec. 5: corrections for an
eps = 0 binary; the 1PN and 2.5PN two-body accelerations in harmonic
coordinates) against facts they must reproduce, not against a retyped formula:

- the jerk is the time derivative of the acceleration along the motion
  (Richardson-extrapolated central differences of the acceleration itself);
- 1PN: an eccentric binary's periastron advances by 6 pi M / (c^2 a (1 - e^2))
  per orbit (Einstein; e.g. Robertson 1938, Damour & Deruelle 1985);
- 2PN: a circular orbit's frequency follows the harmonic-coordinate relation
  omega^2 = (M / r^3) [1 + (-3 + eta) g + (6 + 41/4 eta + eta^2) g^2], g = M / (c^2 r),
  up to terms of order g^3 (residual halving g shrinks 8-fold), which checks the
  terms without rdot; and the 1PN + 2PN equations of motion conserve the 2PN
  two-body energy (the expression in harmonic coordinates, e.g. Blanchet 2014,
  Living Rev. Relativ. 17, 2) up to terms of the next order: its rate of change at
  any phase-space point shrinks as c^-6, where a wrong coefficient of any 2PN term,
  or of the energy, leaves a c^-4 rate;
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


@pytest.mark.parametrize("terms", [oracle.PN_1, oracle.PN_2, oracle.PN_25, oracle.PN_1 | oracle.PN_2 | oracle.PN_25])
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


def _circular_residual(m1, m2, g):
    """Relative radial residual of the Newtonian + 1PN + 2PN acceleration on a circular
    orbit whose frequency comes from the 2PN frequency-separation relation (c = 1)."""
    M = m1 + m2
    eta = m1 * m2 / M ** 2
    r = M / g
    w2 = M / r ** 3 * (1 + (-3 + eta) * g + (6 + 41 / 4 * eta + eta ** 2) * g * g)
    rv = np.array([r, 0.0, 0.0])
    vv = np.array([0.0, np.sqrt(w2) * r, 0.0])
    a = -M * rv / r ** 3 + oracle.pn_accel(m1, m2, rv, vv, 1.0, oracle.PN_1 | oracle.PN_2)
    assert a[1] == 0.0 and a[2] == 0.0  # rdot = 0: no term along v
    return (a[0] + w2 * r) / (w2 * r)


@pytest.mark.parametrize("masses", [(0.5, 0.5), (0.9, 0.1), (0.99, 0.01)])
def test_2pn_circular_orbit_frequency(masses):
    r1 = _circular_residual(*masses, 2e-3)
    r2 = _circular_residual(*masses, 1e-3)
    print("2PN circular orbit residual: g = 2e-3 %.3e, g = 1e-3 %.3e, ratio %.3f" % (r1, r2, r1 / r2))
    # the leftover is the third order: 8x smaller for half the g (a wrong 2PN
    # coefficient would leave a g^2 term: 4x)
    assert 7.5 < r1 / r2 < 8.5
    assert abs(r2) < 1e-7


def _energy_rate(m1, m2, r, v, c, order, terms):
    """d/dt of the two-body energy per reduced mass in harmonic coordinates (through
    1PN or 2PN: v^2/2 - M/r, then 3/8 (1 - 3 eta) v^4 + 1/2 (3 + eta) (M/r) v^2 +
    1/2 eta (M/r) rdot^2 + 1/2 (M/r)^2 over c^2, then the 2PN polynomial below over
    c^4), along the motion r' = v, v' = Newtonian + the oracle's pair terms `terms`,
    by the chain rule through v^2, M/r and rdot."""
    M = m1 + m2
    n = m1 * m2 / M ** 2
    rr = np.linalg.norm(r)
    a = -M * r / rr ** 3 + oracle.pn_accel(m1, m2, r, v, c, terms)
    v2 = v @ v
    rd = r @ v / rr
    Mr = M / rr
    dv2, dMr, drd = 2 * v @ a, -M * rd / rr ** 2, (v2 - rd * rd) / rr + r @ a / rr
    Ev2 = 0.5 + (3 / 4 * (1 - 3 * n) * v2 + 0.5 * (3 + n) * Mr) / c ** 2
    EMr = -1.0 + (0.5 * (3 + n) * v2 + 0.5 * n * rd ** 2 + Mr) / c ** 2
    Erd = n * Mr * rd / c ** 2
    if order >= 2:
        # E2 = 5/16 (1 - 7n + 13n^2) v^6 + 1/8 (21 - 23n - 27n^2) (M/r) v^4
        #      + 1/4 n (1 - 15n) (M/r) v^2 rdot^2 - 3/8 n (1 - 3n) (M/r) rdot^4
        #      + 1/8 (14 - 55n + 4n^2) (M/r)^2 v^2 + 1/8 (4 + 69n + 12n^2) (M/r)^2 rdot^2
        #      - 1/4 (2 + 15n) (M/r)^3
        Ev2 += (15 / 16 * (1 - 7 * n + 13 * n * n) * v2 ** 2 + 1 / 4 * (21 - 23 * n - 27 * n * n) * Mr * v2
                + 1 / 4 * n * (1 - 15 * n) * Mr * rd ** 2 + 1 / 8 * (14 - 55 * n + 4 * n * n) * Mr ** 2) / c ** 4
        EMr += (1 / 8 * (21 - 23 * n - 27 * n * n) * v2 ** 2 + 1 / 4 * n * (1 - 15 * n) * v2 * rd ** 2
                - 3 / 8 * n * (1 - 3 * n) * rd ** 4 + 1 / 4 * (14 - 55 * n + 4 * n * n) * Mr * v2
                + 1 / 4 * (4 + 69 * n + 12 * n * n) * Mr * rd ** 2 - 3 / 4 * (2 + 15 * n) * Mr ** 2) / c ** 4
        Erd += (1 / 2 * n * (1 - 15 * n) * Mr * v2 * rd - 3 / 2 * n * (1 - 3 * n) * Mr * rd ** 3
                + 1 / 4 * (4 + 69 * n + 12 * n * n) * Mr ** 2 * rd) / c ** 4
    return Ev2 * dv2 + EMr * dMr + Erd * drd


def test_2pn_motion_conserves_the_2pn_energy():
    """At random phase-space points and mass ratios the 1PN + 2PN equations of motion
    change the 2PN energy only at the next order: the rate shrinks 64-fold when c
    doubles (c^-6), where the 1PN motion changes the 1PN energy 16-fold (c^-4).  A
    wrong coefficient in any 2PN term of the acceleration (or of the energy) leaves a
    c^-4 rate."""
    rng = np.random.default_rng(11)
    for _ in range(8):
        m1, m2 = rng.uniform(0.02, 1.0, size=2)
        r = rng.normal(size=3)
        v = rng.normal(size=3) * 0.8
        d2 = [_energy_rate(m1, m2, r, v, c, 2, oracle.PN_1 | oracle.PN_2) for c in (100.0, 200.0)]
        d1 = [_energy_rate(m1, m2, r, v, c, 1, oracle.PN_1) for c in (100.0, 200.0)]
        print("energy rates: 2PN %.3e -> %.3e (x%.2f), 1PN x%.4f" % (d2[0], d2[1], d2[0] / d2[1], d1[0] / d1[1]))
        assert 60 < d2[0] / d2[1] < 68
        assert abs(d1[0] / d1[1] - 16) < 1e-3


def test_pn_pair_rejects_bad_arguments():
    m, x, v = _binary(1.0, 0.1)
    sim = oracle.Sim(m, x, v, 0.0, 0.01)
    with pytest.raises(ValueError):
        sim.set_pn(0, 0, 10.0)
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, -1.0)
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, 10.0, terms=8)  # no such term
    sim.set_pn(0, 1, 10.0)
    sim.step()
    with pytest.raises(ValueError):
        sim.set_pn(0, 1, 10.0)  # after the first step
