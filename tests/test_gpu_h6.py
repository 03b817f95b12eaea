"""The sixth-order Hermite GPU path (gd_h6_*, FP64) against the sixth-order
oracle, through the C ABI: force/jerk/snap evaluations, the initial state,
replayed and free-running block schedules, a Kepler binary."""
import numpy as np
import pytest

import oracle
from kepler import kepler_at, kepler_ic
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
ETA6 = 0.2
DT_MIN = 2.0 ** -22


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


def _check(got, want, label):
    for g, w, name in zip(got, want, ("acc", "jerk", "snap")):
        rel = _rel(g, w)
        scale = np.abs(w).max()
        print("%s %s: rel median %.2e p99 %.2e  max|d|/max|w| %.2e" % (label, name, np.median(rel),
                                                                    np.percentile(rel, 99), np.abs(g - w).max() / scale))
        assert np.median(rel) <= 1e-12
        assert np.abs(g - w).max() <= 1e-11 * scale


@pytest.mark.parametrize("n", [1, 2, 3, 127, 1000])
def test_force_jerk_snap_all_active(n):
    """The initial evaluation (a and jerk from the initial state, snap with the
    initial accelerations of all particles) against the oracle's."""
    m, x, v = inputs.plummer(n, seed=n)
    with gravidy.Integrator6(m, x, v, EPS, ETA6) as g:
        st = g.state()
        got = g.force(0, np.arange(n, dtype=np.int32))
    a, j = oracle.force(m, x, v, EPS)
    want = oracle.force6(m, x, v, a, EPS)
    if n > 1:
        _check(got, want, "n=%d" % n)
        _check((st["a"], st["j"], st["s"]), want, "state n=%d" % n)
    else:
        assert np.all(got[0] == 0) and np.all(got[1] == 0) and np.all(got[2] == 0)


@pytest.mark.parametrize("nact", [1, 37, 700, 3000])
def test_force_subsets_and_splits(nact):
    """Active subsets of a power-law sphere (different j-splits), and the same
    particles in another order give the same bits (the split depends only on
    N_act, not on the slot)."""
    n = 3000
    m, x, v = inputs.plummer(n, seed=31, masses=inputs.power_law_masses(n, seed=31))
    idx = inputs.random_subset(n, nact, seed=nact) if nact < n else np.arange(n, dtype=np.int32)
    with gravidy.Integrator6(m, x, v, EPS, ETA6) as g:
        got = g.force(0, idx)
        perm = np.random.default_rng(1).permutation(nact)
        again = g.force(0, idx[perm])
    a, _ = oracle.force(m, x, v, EPS)
    want = oracle.force6(m, x, v, a, EPS, idx)
    _check(got, want, "nact=%d" % nact)
    for q in range(3):
        assert np.array_equal(again[q], got[q][perm])


def test_initial_steps_match_the_oracle():
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim6(m, x, v, EPS, ETA6)
    so = sim.state()
    with gravidy.Integrator6(m, x, v, EPS, ETA6) as g:
        st = g.state()
    assert np.mean(st["dtau"] == so["dtau"]) > 0.99
    assert np.all(st["c"] == 0.0)


def test_replayed_schedule_to_quarter_unit():
    """The oracle's free-running schedule replayed on the GPU: the same block
    times and active lists, so the states agree to round-off growth."""
    m, x, v = inputs.plummer(256, seed=2)
    sim = oracle.Sim6(m, x, v, EPS, ETA6)
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(0.25 / DT_MIN):
            break
    so = sim.state()
    with gravidy.Integrator6(m, x, v, EPS, ETA6) as g:
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
        stats = g.stats()
    dx = np.abs(st["x"] - so["x"]).max()
    dv = np.abs(st["v"] - so["v"]).max()
    print("h6 replay n=256: %d steps, max|dx| %.2e max|dv| %.2e, dtau agree %.4f"
          % (len(rec), dx, dv, np.mean(st["dtau"] == so["dtau"])))
    assert stats["block_steps"] == len(rec)
    assert (st["tau"] == so["tau"]).all()
    assert dx < 1e-9 and dv < 1e-9
    assert np.mean(st["dtau"] == so["dtau"]) > 0.99


def test_free_running_energy_and_schedule_n512_to_t1():
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim6(m, x, v, EPS, ETA6)
    E0 = sum(sim.energy())
    sim.evolve(1.0)
    de_or = abs((sum(sim.energy()) - E0) / E0)
    so = sim.stats()
    with gravidy.Integrator6(m, x, v, EPS, ETA6) as g:
        G0 = sum(g.energy())
        g.evolve(1.0)
        de = abs((sum(g.energy()) - G0) / G0)
        st = g.state()
        stats = g.stats()
    print("h6 free n=512 t=1: blocks %d/%d psteps %d/%d |dE/E| %.3e/%.3e"
          % (stats["block_steps"], so["nblock"], stats["particle_steps"], so["nsteps"], de, de_or))
    assert (st["tau"] == int(1.0 / DT_MIN)).all()
    assert abs(stats["block_steps"] - so["nblock"]) <= 0.01 * so["nblock"]
    assert de <= 2 * de_or + 1e-12


def test_kepler_binary_sixth_order():
    e, t_end = 0.5, 6.25
    m, x, v = kepler_ic(e)
    with gravidy.Integrator6(m, x, v, 0.0, ETA6) as g:
        K0, U0 = g.energy()
        g.evolve(t_end)
        st = g.state()
        K, U = g.energy()
    r = st["x"][1] - st["x"][0]
    r_ex, _ = kepler_at(t_end, e)
    sim = oracle.Sim6(m, x, v, 0.0, ETA6)
    sim.evolve(t_end)
    so = sim.state()
    print("h6 kepler: |dr| %.2e dE/E %.2e vs oracle |dx| %.2e" % (np.abs(r - r_ex).max(), (K + U) / (K0 + U0) - 1,
                                                                 np.abs(st["x"] - so["x"]).max()))
    assert np.abs(r - r_ex).max() < 1e-5
    assert abs((K + U) / (K0 + U0) - 1) < 1e-7
    assert np.abs(st["x"] - so["x"]).max() < 1e-10
