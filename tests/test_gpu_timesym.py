"""The time-symmetric schemes of the gd_h6 engine on the GPU (order 4 with the
time-symmetric corrector, and P(EC)^n passes of either order) against the
oracle, through the C ABI: force and jerk of the order-4 kernel, replayed and
free-running block schedules, and reversibility of the two-pass map on a Kepler
orbit with shared constant steps."""
import numpy as np
import pytest

import oracle
from kepler import kepler_ic
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
ETA4 = 0.01
DT_MIN = 2.0 ** -22


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


@pytest.mark.parametrize("nact", [1, 300, 2000])
def test_order4_force_and_jerk_zero_snap(nact):
    n = 2000
    m, x, v = inputs.plummer(n, seed=41, masses=inputs.power_law_masses(n, seed=41))
    idx = inputs.random_subset(n, nact, seed=nact) if nact < n else np.arange(n, dtype=np.int32)
    with gravidy.Integrator6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4) as g:
        acc, jerk, snap = g.force(0, idx)
        st = g.state()
    a, j = oracle.force(m, x, v, EPS, idx)
    for got, want in ((acc, a), (jerk, j)):
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
    assert np.all(snap == 0.0)
    assert np.all(st["s"] == 0.0) and np.all(st["c"] == 0.0)
    a_all, _ = oracle.force(m, x, v, EPS)
    assert np.abs(st["a"] - a_all).max() <= 1e-11 * np.abs(a_all).max()


@pytest.mark.parametrize("order,n_iter", [(4, 1), (4, 2), (6, 2), (4, 3)])
def test_replayed_schedule(order, n_iter):
    """The oracle's free-running schedule replayed on the GPU: same block times
    and lists, states equal to round-off growth."""
    m, x, v = inputs.plummer(256, seed=3)
    eta, eta_init = (ETA4, ETA4) if order == 4 else (0.2, 0.001)
    sim = oracle.Sim6(m, x, v, EPS, eta, eta_init=eta_init, order=order, n_iter=n_iter)
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(0.25 / DT_MIN):
            break
    so = sim.state()
    sto = sim.stats()
    with gravidy.Integrator6(m, x, v, EPS, eta, eta_init=eta_init, order=order, n_iter=n_iter) as g:
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
        stats = g.stats()
    dx = np.abs(st["x"] - so["x"]).max()
    dv = np.abs(st["v"] - so["v"]).max()
    print("order %d n_iter %d replay n=256: %d steps, max|dx| %.2e max|dv| %.2e, dtau agree %.4f"
          % (order, n_iter, len(rec), dx, dv, np.mean(st["dtau"] == so["dtau"])))
    assert stats["block_steps"] == len(rec)
    assert stats["interactions"] == sto["interactions"]
    assert (st["tau"] == so["tau"]).all()
    assert dx < 1e-9 and dv < 1e-9
    assert np.mean(st["dtau"] == so["dtau"]) > 0.99


@pytest.mark.parametrize("n_iter", [1, 2])
def test_order4_free_run_n512_to_t1(n_iter):
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4, n_iter=n_iter)
    E0 = sum(sim.energy())
    sim.evolve(1.0)
    de_or = abs(sum(sim.energy()) / E0 - 1)
    so = sim.stats()
    with gravidy.Integrator6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4, n_iter=n_iter) as g:
        G0 = sum(g.energy())
        g.evolve(1.0)
        de = abs(sum(g.energy()) / G0 - 1)
        st = g.state()
        stats = g.stats()
    print("order 4 n_iter %d free n=512 t=1: blocks %d/%d psteps %d/%d |dE/E| %.3e/%.3e"
          % (n_iter, stats["block_steps"], so["nblock"], stats["particle_steps"], so["nsteps"], de, de_or))
    assert (st["tau"] == int(1.0 / DT_MIN)).all()
    assert abs(stats["block_steps"] - so["nblock"]) <= 0.01 * so["nblock"]
    assert de <= 2 * de_or + 1e-12


def _kepler_round_trip(order, n_iter, dt=2.0 ** -8, t=6.0):
    """Shared constant steps (dt_min = dt_max = dt) forward to t, velocities
    reversed, forward to t again; returns (distance from the start, the forward
    state, the forward oracle state)."""
    m, x, v = kepler_ic(0.5)
    opts = dict(dt_min=dt, dt_max=dt)
    with gravidy.Integrator6(m, x, v, 0.0, 0.2, order=order, n_iter=n_iter, **opts) as g:
        g.evolve(t)
        fw = g.state()
    with gravidy.Integrator6(m, fw["x"], -fw["v"], 0.0, 0.2, order=order, n_iter=n_iter, **opts) as g:
        g.evolve(t)
        bk = g.state()
    sim = oracle.Sim6(m, x, v, 0.0, 0.2, dt_min=dt, dt_max=dt, order=order, n_iter=n_iter)
    sim.evolve(t)
    return max(np.abs(bk["x"] - x).max(), np.abs(bk["v"] + v).max()), fw, sim.state()


@pytest.mark.parametrize("order", [4, 6])
def test_two_passes_are_reversible_on_the_gpu(order):
    one, fw1, so1 = _kepler_round_trip(order, 1)
    two, fw2, so2 = _kepler_round_trip(order, 2)
    print("GPU order %d round trip: one pass %.2e, two passes %.2e; forward vs oracle %.2e / %.2e"
          % (order, one, two, np.abs(fw1["x"] - so1["x"]).max(), np.abs(fw2["x"] - so2["x"]).max()))
    assert two < 1e-12
    assert one > 30 * two
    for fw, so in ((fw1, so1), (fw2, so2)):
        assert (fw["tau"] == so["tau"]).all()
        assert np.abs(fw["x"] - so["x"]).max() < 1e-11
        assert np.abs(fw["v"] - so["v"]).max() < 1e-11


@pytest.mark.parametrize("order", [4, 6])
def test_single_free_particle_with_the_most_passes(order):
    """One particle (no force): every pass leaves x + v t, exactly, to t = 1/4
    with the largest pass count."""
    m = np.array([1.0])
    x = np.array([[0.25, -0.5, 0.125]])
    v = np.array([[0.5, 0.25, -1.0]])
    with gravidy.Integrator6(m, x, v, EPS, 0.01, order=order, n_iter=16) as g:
        g.evolve(0.25)
        st = g.state()
        stats = g.stats()
    assert (st["tau"] == int(0.25 / DT_MIN)).all()
    assert np.array_equal(st["x"], x + 0.25 * v)
    assert np.array_equal(st["v"], v)
    assert stats["interactions"] == (1 if order == 4 else 2) + 16 * stats["particle_steps"]


def test_three_bodies_sixteen_passes_replay():
    """Pythagorean-like three bodies (masses 3, 4, 5 at the corners of a 3-4-5
    triangle, at rest), eps = 0.01, to t = 8: the oracle's schedule replayed
    with 16 passes per step."""
    m = np.array([3.0, 4.0, 5.0]) / 12.0
    x = np.array([[1.0, 3.0, 0.0], [-2.0, -1.0, 0.0], [1.0, -1.0, 0.0]])
    v = np.zeros((3, 3))
    sim = oracle.Sim6(m, x, v, 0.01, ETA4, eta_init=ETA4, order=4, n_iter=16)
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(8.0 / DT_MIN):
            break
    so = sim.state()
    with gravidy.Integrator6(m, x, v, 0.01, ETA4, eta_init=ETA4, order=4, n_iter=16) as g:
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
    print("three bodies, 16 passes: %d steps, max|dx| %.2e" % (len(rec), np.abs(st["x"] - so["x"]).max()))
    assert (st["tau"] == so["tau"]).all()
    assert np.abs(st["x"] - so["x"]).max() < 1e-11
    assert np.abs(st["v"] - so["v"]).max() < 1e-11


# ---- the time-symmetric corrector on the fourth-order integrator (gd_init, both
# precisions, option corrector = "timesym") against the order-4 oracle with one pass

def _sim4s(m, x, v):
    return oracle.Sim6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4, n_iter=1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_timesym_corrector_replays_the_oracle_schedule_n512_to_t1(prec):
    """The order-4 time-symmetric oracle's free-running schedule replayed on the
    fourth-order GPU integrator with the time-symmetric corrector: FP64 states to
    round-off growth, mixed states to the same bound as the Hermite corrector's
    mixed replay; the energy error against the oracle's."""
    m, x, v = inputs.plummer(512, seed=1)
    sim = _sim4s(m, x, v)
    K0, U0 = sim.energy()
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(1.0 / DT_MIN):
            break
    so = sim.state()
    K1, U1 = sim.energy()
    with gravidy.Integrator(m, x, v, EPS, ETA4, precision=prec, corrector="timesym") as g:
        E0 = sum(g.energy())
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
        E1 = sum(g.energy())
    de_or = (K1 + U1 - K0 - U0) / (K0 + U0)
    de = (E1 - E0) / E0
    dx = np.abs(st["x"] - so["x"]).max()
    agree = np.mean(st["dtau"] == so["dtau"])
    print("%s timesym replay n=512: %d steps |dE/E| oracle %.3e gpu %.3e max|dx| %.2e dtau agree %.4f"
          % (prec, len(rec), abs(de_or), abs(de), dx, agree))
    assert (st["tau"] == so["tau"]).all()
    if prec == "fp64":
        assert dx < 1e-9 and abs(de - de_or) < 1e-10 and agree > 0.99
    else:
        assert dx < 1e-4 and abs(de) < 2 * abs(de_or) + 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_timesym_corrector_free_run_n512_to_t1(prec):
    """Free run to t = 1 with the time-symmetric corrector: block and particle
    step counts of the order-4 time-symmetric oracle (identical for FP64 up to a
    quantisation decision at a boundary, within 1 % for the mixed path) and an
    energy error within 2x of the oracle's."""
    m, x, v = inputs.plummer(512, seed=1)
    sim = _sim4s(m, x, v)
    K0, U0 = sim.energy()
    sim.evolve(1.0)
    K1, U1 = sim.energy()
    so = sim.stats()
    de_or = abs((K1 + U1 - K0 - U0) / (K0 + U0))
    with gravidy.Integrator(m, x, v, EPS, ETA4, precision=prec, corrector="timesym") as g:
        E0 = sum(g.energy())
        g.evolve(1.0)
        de = abs((sum(g.energy()) - E0) / E0)
        st = g.stats()
    print("%s timesym free n=512 t=1: |dE/E| oracle %.3e gpu %.3e blocks %d/%d psteps %d/%d"
          % (prec, de_or, de, st["block_steps"], so["nblock"], st["particle_steps"], so["nsteps"]))
    tol = 0.002 if prec == "fp64" else 0.01
    assert abs(st["block_steps"] - so["nblock"]) <= tol * so["nblock"]
    assert abs(st["particle_steps"] - so["nsteps"]) <= tol * so["nsteps"]
    assert de <= 2 * de_or + 1e-9


@pytest.mark.parametrize("opts", [dict(cluster=False), dict(fused=True)])
def test_timesym_corrector_paths_agree(opts):
    """The small-step cluster (default) against every step on the full GPU (force
    sums in another order: round-off growth), and the fused cooperative kernel
    (the same arithmetic: bit-identical), with the time-symmetric corrector."""
    m, x, v = inputs.plummer(3000, seed=17)
    res = []
    for o in (dict(), opts):
        with gravidy.Integrator(m, x, v, EPS, ETA4, precision="mixed", corrector="timesym", **o) as g:
            g.evolve(0.125)
            res.append(g.state())
    a, b = res
    if opts.get("fused"):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    else:
        assert (a["tau"] == b["tau"]).all()
        assert np.mean(a["dtau"] == b["dtau"]) > 0.99
        assert np.abs(a["x"] - b["x"]).max() < 1e-6


def test_timesym_corrector_in_an_ensemble_follows_each_cluster_alone():
    sizes = [300, 777, 64]
    ms, xs, vs = [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(n, seed=500 + q)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA4,
                          corrector="timesym") as e:
        e.evolve(0.25)
        st = e.state()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for q, n in enumerate(sizes):
        with gravidy.Integrator(ms[q], xs[q], vs[q], EPS, ETA4, precision="mixed", corrector="timesym") as g:
            g.evolve(0.25)
            so = g.state()
        sl = slice(off[q], off[q + 1])
        assert np.mean(st["dtau"][sl] == so["dtau"]) > 0.99
        assert np.abs(st["x"][sl] - so["x"]).max() < 1e-6


# ---- P(EC)^n passes on the fourth-order integrator (gd_init, gd_opts.n_iter, with
# the time-symmetric corrector) against the order-4 oracle with the same passes

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n_iter", [2, 3])
def test_passes_replay_the_oracle_schedule_n512(prec, n_iter):
    """The oracle's free-running P(EC)^n schedule replayed on the fourth-order GPU
    integrator with the same passes: FP64 states to round-off growth, mixed states
    within the bound of the one-pass mixed replay; every pass counts its
    interactions."""
    m, x, v = inputs.plummer(512, seed=2)
    sim = oracle.Sim6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4, n_iter=n_iter)
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(0.5 / DT_MIN):
            break
    so = sim.state()
    with gravidy.Integrator(m, x, v, EPS, ETA4, precision=prec, corrector="timesym", n_iter=n_iter,
                            cluster=False) as g:
        i0 = g.stats()["interactions"]
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
        inter = g.stats()["interactions"] - i0
    dx = np.abs(st["x"] - so["x"]).max()
    print("%s n_iter %d replay n=512: %d steps, max|dx| %.2e, dtau agree %.4f"
          % (prec, n_iter, len(rec), dx, np.mean(st["dtau"] == so["dtau"])))
    assert inter == n_iter * 512.0 * sum(len(idx) for _, idx in rec)
    assert (st["tau"] == so["tau"]).all()
    if prec == "fp64":
        assert dx < 1e-9 and np.mean(st["dtau"] == so["dtau"]) > 0.99
    else:
        assert dx < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_passes_free_run_n512_to_t1(prec):
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim6(m, x, v, EPS, ETA4, eta_init=ETA4, order=4, n_iter=2)
    K0, U0 = sim.energy()
    sim.evolve(1.0)
    K1, U1 = sim.energy()
    so = sim.stats()
    de_or = abs((K1 + U1 - K0 - U0) / (K0 + U0))
    with gravidy.Integrator(m, x, v, EPS, ETA4, precision=prec, corrector="timesym", n_iter=2) as g:
        E0 = sum(g.energy())
        g.evolve(1.0)
        de = abs((sum(g.energy()) - E0) / E0)
        st = g.stats()
    print("%s n_iter 2 free n=512 t=1: |dE/E| oracle %.3e gpu %.3e blocks %d/%d psteps %d/%d"
          % (prec, de_or, de, st["block_steps"], so["nblock"], st["particle_steps"], so["nsteps"]))
    tol = 0.002 if prec == "fp64" else 0.01
    assert abs(st["block_steps"] - so["nblock"]) <= tol * so["nblock"]
    assert abs(st["particle_steps"] - so["nsteps"]) <= tol * so["nsteps"]
    assert de <= 2 * de_or + 1e-9


def test_two_passes_reversible_on_the_fourth_order_integrator():
    """Shared constant steps on a Kepler orbit (FP64): forward to t = 6, velocities
    reversed, forward again; two passes return to the start to round-off, one pass
    does not (its map is not time-symmetric)."""
    dt = 2.0 ** -8
    m, x, v = kepler_ic(0.5)
    err = {}
    for n_iter in (1, 2):
        kw = dict(precision="fp64", corrector="timesym", n_iter=n_iter, dt_min=dt, dt_max=dt)
        with gravidy.Integrator(m, x, v, 0.0, 0.2, **kw) as g:
            g.evolve(6.0)
            fw = g.state()
        with gravidy.Integrator(m, fw["x"], -fw["v"], 0.0, 0.2, **kw) as g:
            g.evolve(6.0)
            bk = g.state()
        err[n_iter] = max(np.abs(bk["x"] - x).max(), np.abs(bk["v"] + v).max())
    print("fourth-order integrator Kepler round trip: one pass %.2e, two passes %.2e" % (err[1], err[2]))
    assert err[2] < 1e-12
    assert err[1] > 30 * err[2]


def test_two_passes_in_the_small_step_cluster_and_on_the_full_gpu():
    """P(EC)^2 through the small-step cluster (trial records rewritten in shared memory
    and gathered again) against every step on the full GPU: the same arithmetic, force
    sums in another order, so the runs agree to round-off growth."""
    m, x, v = inputs.plummer(3000, seed=23)
    out = []
    for cl in (True, False):
        with gravidy.Integrator(m, x, v, EPS, ETA4, precision="mixed", corrector="timesym", n_iter=2,
                                cluster=cl) as g:
            assert (g.cluster_info()[0] > 0) == cl
            g.evolve(0.125)
            out.append((g.state(), g.stats()))
    (a, sa), (b, sb) = out
    print("n_iter 2 cluster vs full GPU: psteps %d / %d, dtau agree %.4f, max|dx| %.2e"
          % (sa["particle_steps"], sb["particle_steps"], np.mean(a["dtau"] == b["dtau"]), np.abs(a["x"] - b["x"]).max()))
    assert (a["tau"] == b["tau"]).all()
    assert np.mean(a["dtau"] == b["dtau"]) > 0.99
    assert np.abs(a["x"] - b["x"]).max() < 1e-6
    assert abs(sa["particle_steps"] - sb["particle_steps"]) <= 0.01 * sb["particle_steps"]
    assert abs(sa["interactions"] / sb["interactions"] - 1) < 0.01
