"""Ensembles of independent clusters (gd_ens_*) against single-system runs of
each cluster and against the oracle.

A cluster in an ensemble follows the same scheme as the cluster alone; only
the j-split of the force sums (so the last bits of the forces) differs, so the
block schedules agree and the states agree to round-off growth over the run.
"""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
ETA = 0.01
U32 = 2.0 ** -24
SIZES = [200, 300, 513, 129, 64, 777]


def _clusters(sizes, seed0=100):
    ms, xs, vs = [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(n, seed=seed0 + q)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    return ms, xs, vs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def test_ensemble_energy_matches_oracle_per_cluster():
    ms, xs, vs = _clusters(SIZES)
    with gravidy.Ensemble(SIZES, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA) as e:
        K, U = e.energy()
    for q in range(len(SIZES)):
        Ko, Uo = oracle.energy(ms[q], xs[q], vs[q], EPS)
        assert K[q] == pytest.approx(Ko, rel=1e-13)
        assert U[q] == pytest.approx(Uo, rel=8 * U32)


def test_ensemble_follows_each_cluster_alone():
    ms, xs, vs = _clusters(SIZES)
    t_end = 0.25
    with gravidy.Ensemble(SIZES, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA) as e:
        K0, U0 = e.energy()
        e.evolve(t_end)
        K1, U1 = e.energy()
        st = e.state()
        es = e.stats()
    off = np.concatenate([[0], np.cumsum(SIZES)])
    psteps = 0
    for q, n in enumerate(SIZES):
        sl = slice(off[q], off[q + 1])
        with gravidy.Integrator(ms[q], xs[q], vs[q], EPS, ETA, precision="mixed") as g:
            g.evolve(t_end)
            so = g.state()
            psteps += g.stats()["particle_steps"]
        agree = np.mean(st["dtau"][sl] == so["dtau"])
        dx = np.abs(st["x"][sl] - so["x"]).max()
        assert (st["tau"][sl] == int(t_end / 2.0 ** -22)).all()
        assert agree > 0.99, agree
        assert dx < 1e-6, dx
        # energy error of the cluster vs the oracle's for the same cluster
        sim = oracle.Sim(ms[q], xs[q], vs[q], EPS, ETA)
        Ko, Uo = sim.energy()
        sim.evolve(t_end)
        Ko1, Uo1 = sim.energy()
        de_or = abs((Ko1 + Uo1 - Ko - Uo) / (Ko + Uo))
        de = abs((K1[q] + U1[q] - K0[q] - U0[q]) / (K0[q] + U0[q]))
        print("cluster %d n=%d: dtau agree %.4f max|dx| %.1e |dE/E| ens %.2e oracle %.2e" % (q, n, agree, dx, de, de_or))
        assert de <= 2 * de_or + 2e-9
    # the ensemble's particle steps are the clusters' particle steps
    assert abs(es["particle_steps"] - psteps) <= 0.01 * psteps


def test_ensemble_block_steps_interleave():
    ms, xs, vs = _clusters([256, 1000], seed0=7)
    with gravidy.Ensemble([256, 1000], np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA) as e:
        last = 0.0
        for _ in range(200):
            t, nact = e.step_block()
            assert t > last and nact >= 1
            last = t
        st = e.state()
    assert (st["tau"] % st["dtau"] == 0).all()
    assert ((st["dtau"] & (st["dtau"] - 1)) == 0).all()


def test_ensemble_rejects_fp64_and_bad_sizes():
    m, x, v = inputs.plummer(64, seed=1)
    with pytest.raises(gravidy.GravidyError):
        gravidy.Ensemble([64], m, x, v, EPS, ETA, precision="fp64")
    with pytest.raises(gravidy.GravidyError):
        gravidy.Ensemble([0, 64], m, x, v, EPS, ETA)


@pytest.mark.parametrize("steps_per_launch", [1, 16])
def test_fused_ensemble_launches_match_the_two_kernel_steps(steps_per_launch):
    """The cooperative ensemble kernel (select, grid barrier, force + correction,
    grid barrier per global block step; one launch per step or sixteen steps per
    launch) takes the same steps with the same arithmetic as the two-kernel graph:
    bit-identical states and counters."""
    sizes = [300, 1000, 64, 2500, 777]
    ms, xs, vs = _clusters(sizes, seed0=300)
    out = []
    for opts in (dict(cluster=False), dict(fused=True, graph_steps=steps_per_launch)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(0.25)
            st = e.state()
            s = e.stats()
            st["stats"] = np.array([s["tick"], s["block_steps"], s["particle_steps"]])
            st["K"], st["U"] = e.energy()
            out.append(st)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("t_end", [0.125, 0.375])
def test_independent_systems_follow_the_global_steps(t_end):
    """Each system integrated to the end inside its own thread-block cluster (the
    default ensemble path) against the global-block-time two-kernel path: the same
    scheme and arithmetic per particle, force sums split over other CTAs, so the
    runs agree to round-off growth.  The sizes include a three-body system (CTAs
    without particles), systems whose steps take more active particles than one
    batch, and one whose CTAs own more active particles than their outbox holds."""
    sizes = [2500, 3, 700, 129, 1500, 64]
    ms, xs, vs = _clusters(sizes, seed0=500)
    out = []
    for opts in (dict(), dict(cluster=False)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(t_end)
            st = e.state()
            s = e.stats()
            K, U = e.energy()
            out.append((st, s, K + U))
    (a, sa, Ea), (b, sb, Eb) = out
    print("systems vs global: psteps %d / %d, dtau agree %.4f, max|dx| %.2e, max rel dE %.2e"
          % (sa["particle_steps"], sb["particle_steps"], np.mean(a["dtau"] == b["dtau"]),
             np.abs(a["x"] - b["x"]).max(), np.max(np.abs(Ea - Eb) / np.abs(Eb))))
    tick = int(t_end / 2.0 ** -22)
    assert (a["tau"] == tick).all() and (b["tau"] == tick).all()
    assert np.mean(a["dtau"] == b["dtau"]) > 0.99
    assert np.abs(a["x"] - b["x"]).max() < 1e-6
    assert abs(sa["particle_steps"] - sb["particle_steps"]) <= 0.01 * sb["particle_steps"]
    assert abs(sa["interactions"] - sb["interactions"]) <= 0.01 * sb["interactions"]
    assert np.all(np.abs(Ea - Eb) <= 1e-6 * np.abs(Eb))


def test_independent_systems_then_global_steps():
    """The state after the independent-systems path continues on the global path
    (step_block) at the next block time of all systems."""
    sizes = [300, 1000]
    ms, xs, vs = _clusters(sizes, seed0=9)
    with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA) as e:
        e.evolve(0.125)
        st = e.state()
        t, nact = e.step_block()
    assert t > 0.125 and nact >= 1
    assert t == 0.125 + st["dtau"].min() * 2.0 ** -22


def test_independent_systems_with_a_sixteen_cta_cluster():
    """A cluster of 11000 particles needs the 16-CTA class (more than 8 x 1280), a
    small one the 1-CTA class: both against the global two-kernel path."""
    sizes = [11000, 500]
    ms, xs, vs = _clusters(sizes, seed0=700)
    out = []
    for opts in (dict(), dict(cluster=False)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(0.125)
            out.append((e.state(), e.stats()))
    (a, sa), (b, sb) = out
    print("16-CTA class: psteps %d / %d, dtau agree %.4f, max|dx| %.2e"
          % (sa["particle_steps"], sb["particle_steps"], np.mean(a["dtau"] == b["dtau"]), np.abs(a["x"] - b["x"]).max()))
    assert (a["tau"] == b["tau"]).all()
    assert np.mean(a["dtau"] == b["dtau"]) > 0.99
    assert np.abs(a["x"] - b["x"]).max() < 1e-6
    assert abs(sa["particle_steps"] - sb["particle_steps"]) <= 0.01 * sb["particle_steps"]


def test_independent_systems_at_the_class_edges_and_the_size_limit():
    """Clusters of exactly 1280, 1281 and 20480 particles (a full 1-CTA cluster, the
    smallest 2-CTA one, a full 16-CTA one) against the global path; an ensemble with
    a cluster above 16 x 1280 particles falls back to the global path as a whole."""
    sizes = [1280, 1281, 20480]
    ms, xs, vs = _clusters(sizes, seed0=800)
    out = []
    for opts in (dict(), dict(cluster=False)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(0.125)
            out.append((e.state(), e.stats()))
    (a, sa), (b, sb) = out
    assert (a["tau"] == b["tau"]).all()
    assert np.mean(a["dtau"] == b["dtau"]) > 0.99
    assert np.abs(a["x"] - b["x"]).max() < 1e-6
    assert abs(sa["particle_steps"] - sb["particle_steps"]) <= 0.01 * sb["particle_steps"]
    sizes = [21000, 100]
    ms, xs, vs = _clusters(sizes, seed0=900)
    res = []
    for opts in (dict(), dict(cluster=False)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(0.125)
            res.append(e.state())
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]), k


def test_independent_systems_to_an_end_time_between_synchronisations():
    """t_end not a multiple of dt_max: every particle stops at its last step at or
    before t_end, as on the global path, and the next global block step is the
    earliest next time of the state left behind."""
    sizes = [700, 1500, 40]
    ms, xs, vs = _clusters(sizes, seed0=950)
    out = []
    for opts in (dict(), dict(cluster=False)):
        with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                              **opts) as e:
            e.evolve(0.3)
            st = e.state()
            t_next, _ = e.step_block()
            out.append((st, t_next))
    (a, ta), (b, tb) = out
    assert np.mean(a["tau"] == b["tau"]) > 0.99
    assert a["tau"].max() <= int(0.3 / 2.0 ** -22)
    assert np.mean(a["dtau"] == b["dtau"]) > 0.99
    same = a["tau"] == b["tau"]  # particles at the same time (a flipped step moves the rest)
    assert np.abs(a["x"][same] - b["x"][same]).max() < 1e-6
    for st, t in ((a, ta), (b, tb)):
        assert t == (st["tau"] + st["dtau"]).min() * 2.0 ** -22
