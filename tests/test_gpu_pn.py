"""Post-Newtonian pair terms on the GPU (gd_opts.pn_*; Sec. 5's corrections for
a binary) against the oracle's, through the C ABI: the force hook, a replayed
block schedule of a binary in a small cluster, and the periastron advance of an
isolated binary under the integrator's own block steps."""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS, ETA = 1e-4, 0.01
DT_MIN = 2.0 ** -22
U24 = 2.0 ** -24
PN_ALL = gravidy.GD_PN_1 | gravidy.GD_PN_2 | gravidy.GD_PN_25


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def _binary(m1, m2, a, e):
    M = m1 + m2
    r = np.array([a * (1 - e), 0.0, 0.0])
    v = np.array([0.0, np.sqrt(M * (1 + e) / (a * (1 - e))), 0.0])
    return np.array([m1, m2]), np.stack([m2 / M * r, -m1 / M * r]), np.stack([m2 / M * v, -m1 / M * v])


def _cluster_with_binary(nfield=62, seed=5):
    """A binary (0.3 + 0.2, a = 0.02, e = 0.4) at the centre of a Plummer sphere
    of nfield particles of total mass 0.5."""
    mb, xb, vb = _binary(0.3, 0.2, 0.02, 0.4)
    mf, xf, vf = inputs.plummer(nfield, seed=seed)
    return np.concatenate([mb, 0.5 * mf]), np.concatenate([xb, xf]), np.concatenate([vb, vf])


def _pn_share(m, x, v, p, q, c, terms, i):
    r, vr = x[p] - x[q], v[p] - v[q]
    M = m[p] + m[q]
    ar = -M * r / np.linalg.norm(r) ** 3
    w = m[q] / M if i == p else -m[p] / M
    return w * oracle.pn_accel(m[p], m[q], r, vr, c, terms), w * oracle.pn_jerk(m[p], m[q], r, vr, ar, c, terms)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("terms", [gravidy.GD_PN_1, gravidy.GD_PN_2, gravidy.GD_PN_25, PN_ALL])
def test_pn_force_hook_matches_the_oracle(prec, terms):
    m, x, v = _cluster_with_binary()
    c = 30.0
    idx = np.arange(m.size, dtype=np.int32)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, pn=(0, 1, c, terms)) as g:
        a, j = g.force(0, idx)
    a_or, j_or = oracle.force(m, x, v, EPS, idx)
    an, jn = oracle.force_absnorm(m, x, v, EPS, idx)
    for i in (0, 1):
        da, dj = _pn_share(m, x, v, 0, 1, c, terms, i)
        a_or[i] += da
        j_or[i] += dj
    # FP64: round-off of the sums and of the pair terms; mixed: the force's term
    # bound plus FP32 pair terms (a few units of 2^-24 of their own size)
    tol = 1e-12 if prec == "fp64" else 16 * U24
    pn_a = np.abs(_pn_share(m, x, v, 0, 1, c, terms, 0)[0]).max()
    assert (np.abs(a - a_or).max(axis=1) <= tol * (an + pn_a)).all()
    assert (np.abs(j - j_or).max(axis=1) <= tol * (jn + np.abs(_pn_share(m, x, v, 0, 1, c, terms, 0)[1]).max())).all()
    # the pair terms are really there: they move the pair's force by far more than the tolerance
    assert pn_a > 10 * tol * an[0]


def _record(sim, t_end):
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(t_end / DT_MIN):
            return rec


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pn_replayed_schedule_matches_the_oracle(prec):
    """The oracle's free-running schedule of the binary in its cluster (about ten
    binary orbits) replayed on the GPU with the same pair terms."""
    m, x, v = _cluster_with_binary()
    c = 30.0
    sim = oracle.Sim(m, x, v, EPS, ETA)
    sim.set_pn(0, 1, c, PN_ALL)
    rec = _record(sim, 0.25)
    so = sim.state()
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, pn=(0, 1, c, PN_ALL)) as g:
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
    dx = np.abs(st["x"] - so["x"]).max()
    rb = np.linalg.norm(so["x"][0] - so["x"][1])
    dxb = np.linalg.norm((st["x"][0] - st["x"][1]) - (so["x"][0] - so["x"][1]))
    print("%s pn replay: %d steps, max|dx| %.2e, binary separation %.3e off by %.2e" % (prec, len(rec), dx, rb, dxb))
    assert (st["tau"] == so["tau"]).all()
    if prec == "fp64":
        assert dx < 1e-9
    else:
        assert dx < 1e-4 and dxb < 1e-3 * rb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("terms", [gravidy.GD_PN_1, gravidy.GD_PN_1 | gravidy.GD_PN_2])
def test_pn_periastron_advance_under_block_steps(prec, terms):
    """An isolated eccentric binary (eps = 0) integrated by gd_evolve with the
    1PN (and 2PN) terms: its periastron advances by 6 pi M / (c^2 a (1 - e^2)) per
    orbit, to within 1 % at M / (c^2 a) = 1.1e-3 (the formula's own next order,
    where the 2PN terms act), as the oracle's free run with the same block steps
    and terms does."""
    a, e, c = 1.0, 0.5, 30.0
    m, x, v = _binary(0.6, 0.4, a, e)
    M = m.sum()
    period = 2 * np.pi * np.sqrt(a ** 3 / M)
    dt_max = 2.0 ** -9

    def advance(states):
        rs = np.array([s[0] - s[1] for s in states])
        rr = np.linalg.norm(rs, axis=1)
        ang = np.unwrap(np.arctan2(rs[:, 1], rs[:, 0]))
        peri = []
        for k in range(1, rr.size - 1):
            if rr[k] < rr[k - 1] and rr[k] <= rr[k + 1]:
                y0, y1, y2 = rr[k - 1], rr[k], rr[k + 1]
                s = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
                a0, a1, a2 = ang[k - 1], ang[k], ang[k + 1]
                peri.append(a1 + s * 0.5 * (a2 - a0) + s * s * 0.5 * (a2 - 2 * a1 + a0))
        return (np.diff(peri) - 2 * np.pi).mean()

    # sample both runs at the same times: every dt_max (all particles synchronised)
    t_samples = np.arange(1, int(6 * period / dt_max)) * dt_max
    with gravidy.Integrator(m, x, v, 0.0, ETA, precision=prec, dt_max=dt_max, pn=(0, 1, c, terms)) as g:
        gs = []
        for t in t_samples:
            g.evolve(t)
            gs.append(g.state()["x"])
    sim = oracle.Sim(m, x, v, 0.0, ETA, dt_max=dt_max)
    sim.set_pn(0, 1, c, terms)
    os_ = []
    for t in t_samples:
        sim.evolve(t)
        os_.append(sim.state()["x"])
    want = 6 * np.pi * M / (c * c * a * (1 - e * e))
    got_g, got_o = advance(gs), advance(os_)
    print("%s pn %d periastron advance per orbit: gpu %.5e oracle %.5e formula %.5e" % (prec, terms, got_g, got_o, want))
    assert abs(got_o / want - 1) < 0.01
    assert abs(got_g / want - 1) < 0.01
    assert abs(got_g / got_o - 1) < (1e-6 if prec == "fp64" else 2e-3)


def test_pn_small_step_cluster_and_full_gpu_agree():
    """The binary in its cluster, free-running with all three orders on: the
    small-step cluster (pair terms from both members' records in distributed shared
    memory) against every step on the full GPU; the same arithmetic, force sums in
    another order, so the runs agree to round-off growth."""
    m, x, v = _cluster_with_binary()
    c = 30.0
    out = []
    for cl in (True, False):
        with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", cluster=cl, pn=(0, 1, c, PN_ALL)) as g:
            assert (g.cluster_info()[0] > 0) == cl
            g.evolve(0.125)
            out.append((g.state(), g.stats()))
    (a, sa), (b, sb) = out
    rb = np.linalg.norm(b["x"][0] - b["x"][1])
    dxb = np.linalg.norm((a["x"][0] - a["x"][1]) - (b["x"][0] - b["x"][1]))
    print("pn cluster vs full GPU: psteps %d / %d, max|dx| %.2e, binary separation off by %.2e of %.3e"
          % (sa["particle_steps"], sb["particle_steps"], np.abs(a["x"] - b["x"]).max(), dxb, rb))
    assert (a["tau"] == b["tau"]).all()
    assert np.mean(a["dtau"] == b["dtau"]) > 0.98
    assert np.abs(a["x"] - b["x"]).max() < 1e-4 and dxb < 1e-3 * rb
    assert abs(sa["particle_steps"] - sb["particle_steps"]) <= 0.01 * sb["particle_steps"]
