"""GPU path vs the FP64 oracle, through the C ABI (ctypes binding).

Tolerances:
  FP64 path   per-particle |a_gpu - a_oracle| / |a| <= 1e-12 (force/jerk), plus a
              round-off bound scaled by the sum of term magnitudes.
  mixed path  FP32 pair arithmetic on double-single positions (m / s^3 with one
              Newton step on rsqrt.approx), FP32 sums over the terms of one j-tile
              folded into compensated sums.  Per component the error stays below
              16 units of 2^-24 times sum_j |term_j| (measured at most 8 units: a term
              carries a few units from the difference, r^2, the refined rsqrt and the
              products, and a tile's FP32 sum adds rounding errors that mostly
              cancel).  Per particle, |a_gpu - a_oracle| / |a| and the same for the
              jerk are held to <= 1e-6 at the median and, over sets of at least 200
              particles, at the 99th percentile.  The largest per-particle errors
              belong to particles whose terms cancel (sum_j |term_j| / |jerk| up to
              about 700): measured up to 1.1e-6 for a and 1.1e-5 for the jerk; the
              per-component bound above holds for them too.
"""
import numpy as np
import pytest

import oracle
from paper_1702_00440_gb300 import gravidy, inputs

pytestmark = pytest.mark.gpu

EPS = 1e-4
ETA = 0.01
DT_MIN = 2.0 ** -22
U32 = 2.0 ** -24
MIXED_TERM_BOUND = 16 * U32
# the mixed path's 99th percentile of |d jerk| / |jerk| for power-law masses (dN/dm ~ m^-2.35
# over a factor 100): measured 1.0-1.07e-6 at N = 5000, against 0.65-0.9e-6 for equal masses
POWER_LAW_JERK_P99 = 1.5e-6


def fp64_term_bound(n):
    """FP64 path: sums of up to n terms, each with a few ulp of its own error;
    the summation error of n terms with independent roundings stays below about
    8 sqrt(n) units with overwhelming probability (probabilistic bound of Higham
    and Mary for recursive summation), plus the per-term part."""
    return (16 + 8 * n ** 0.5) * 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


def _check_force(prec, m, x, v, eps, idx, label="", jerk_p99=1e-6, **opts):
    n = m.shape[0]
    with gravidy.Integrator(m, x, v, eps, ETA, precision=prec, **opts) as g:
        a, j = g.force(0, idx)
    a_or, j_or = oracle.force(m, x, v, eps, idx)
    an, jn = oracle.force_absnorm(m, x, v, eps, idx)
    bound = MIXED_TERM_BOUND if prec == "mixed" else fp64_term_bound(m.size)
    ra = np.abs(a - a_or).max(axis=1) / an
    rj = np.abs(j - j_or).max(axis=1) / jn
    rel_a = np.linalg.norm(a - a_or, axis=1) / np.linalg.norm(a_or, axis=1)
    rel_j = np.linalg.norm(j - j_or, axis=1) / np.linalg.norm(j_or, axis=1)
    print("%s %s n=%d nact=%d: max|da|/sum|a_j| %.2e max|dj|/sum|j_j| %.2e  rel a med %.2e p99 %.2e max %.2e"
          "  rel j med %.2e p99 %.2e max %.2e" % (label, prec, n, idx.size, ra.max(), rj.max(), np.median(rel_a),
                                                np.percentile(rel_a, 99), rel_a.max(), np.median(rel_j),
                                                np.percentile(rel_j, 99), rel_j.max()))
    assert ra.max() <= bound
    assert rj.max() <= bound
    if prec == "fp64":
        assert np.median(rel_a) <= 1e-12 and np.median(rel_j) <= 1e-12
        assert np.percentile(rel_a, 99) <= 1e-12
    else:
        assert np.median(rel_a) <= 1e-6 and np.median(rel_j) <= 1e-6
        if idx.size >= 200:
            assert np.percentile(rel_a, 99) <= 1e-6 and np.percentile(rel_j, 99) <= jerk_p99


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 3, 127, 512, 1000, 3001])
def test_force_all_active(prec, n):
    m, x, v = inputs.plummer(n, seed=n)
    if n < 3:
        x = x + np.arange(3 * n).reshape(n, 3) * 0.1  # distinct points
    idx = np.arange(n, dtype=np.int32)
    if n == 1:
        with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec) as g:
            a, j = g.force(0, idx)
        assert np.array_equal(a, np.zeros((1, 3))) and np.array_equal(j, np.zeros((1, 3)))
        return
    _check_force(prec, m, x, v, EPS, idx, label="all")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nact", [1, 5, 32, 33, 191, 192, 257, 700, 2049])
@pytest.mark.parametrize("mode_cut", [1, 10 ** 9])
def test_force_subsets_split(prec, nact, mode_cut):
    """Both work decompositions (mode_cut 1: i-parallel tiles always; 10^9:
    warp tiles always) with the automatic j-split; ragged N spans several
    j-tiles and a padded tail."""
    n = 5000
    m, x, v = inputs.plummer(n, seed=7, masses=inputs.power_law_masses(n, seed=7))
    idx = inputs.random_subset(n, nact, seed=nact)
    # power-law masses: the mixed jerk's tail of cancelling sums reaches about 1.1e-6 at p99
    _check_force(prec, m, x, v, EPS, idx, label="subset mc=%d" % mode_cut, jerk_p99=POWER_LAW_JERK_P99,
                 mode_cut=mode_cut)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("jsplit", [1, 3, 19, 40])
@pytest.mark.parametrize("nact", [1, 9, 300])
def test_force_forced_split_factors(prec, jsplit, nact):
    """Forced j-split factors: the last CTA of each i-tile sums S partials,
    with one or several threads per (slot, component)."""
    n = 10000
    m, x, v = inputs.plummer(n, seed=17)
    idx = inputs.random_subset(n, nact, seed=jsplit)
    _check_force(prec, m, x, v, EPS, idx, label="S=%d" % jsplit, jsplit=jsplit)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotuned_table_keeps_parity(prec):
    n = 6000
    m, x, v = inputs.plummer(n, seed=23)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, autotune=True) as g:
        mc, split, mode, ms = g.tuning()
        print("%s tuning: split %s mode %s" % (prec, split[:14].tolist(), mode[:14].tolist()))
        assert (mode[:12] >= 0).all() and (split[:12] > 0).all()
        for nact in (1, 7, 64, 900, n):
            idx = inputs.random_subset(n, nact, seed=nact)
            a, j = g.force(0, idx)
            a_or, j_or = oracle.force(m, x, v, EPS, idx)
            an, jn = oracle.force_absnorm(m, x, v, EPS, idx)
            bound = MIXED_TERM_BOUND if prec == "mixed" else fp64_term_bound(m.size)
            assert (np.abs(a - a_or).max(axis=1) <= bound * an).all()
            assert (np.abs(j - j_or).max(axis=1) <= bound * jn).all()
        g.evolve(0.125)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_force_unsoftened(prec):
    m, x, v = inputs.plummer(700, seed=3)
    idx = np.arange(700, dtype=np.int32)
    _check_force(prec, m, x, v, 0.0, idx, label="eps0")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_force_duplicates_and_order(prec):
    m, x, v = inputs.plummer(300, seed=5)
    idx = np.array([7, 3, 3, 299, 0, 7], dtype=np.int32)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec) as g:
        a, j = g.force(0, idx)
    assert np.array_equal(a[1], a[2]) and np.array_equal(a[0], a[5])
    a_or, _ = oracle.force(m, x, v, EPS, idx)
    np.testing.assert_allclose(a, a_or, rtol=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nact", [3, 13, 300, 777])
@pytest.mark.parametrize("mode_cut", [1, 10 ** 9])
def test_force_independent_of_slot(prec, nact, mode_cut):
    """A particle's force is bit-identical wherever it sits in the active list
    (the free-running step lists active particles in the order their chunks
    claim places, not ascending): permuting the list permutes the results."""
    n = 5000
    m, x, v = inputs.plummer(n, seed=21)
    idx = inputs.random_subset(n, nact, seed=nact)
    perm = np.random.default_rng(nact).permutation(nact)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, mode_cut=mode_cut) as g:
        a, j = g.force(0, idx)
        ap, jp = g.force(0, idx[perm])
    assert np.array_equal(ap, a[perm]) and np.array_equal(jp, j[perm])


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    m, x, v = inputs.plummer(n, seed=seed)
    a = rng.normal(size=(n, 3))
    j = rng.normal(size=(n, 3)) * 3
    dtau = 2 ** rng.integers(0, 8, size=n).astype(np.int64) * 64
    tau = (rng.integers(0, 40, size=n).astype(np.int64) * dtau)
    return m, x, v, a, j, tau, dtau


def test_predictor_matches_oracle():
    n = 1537
    m, x, v, a, j, tau, dtau = _random_state(n, 3)
    tick = int((tau + dtau).max())
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        g.set_state(x, v, a, j, tau, dtau)
        xp, vp = g.predict(tick)
    for i in range(n):
        dt = (tick - tau[i]) * DT_MIN
        xo, vo = oracle.predict_one(x[i], v[i], a[i], j[i], dt)
        scale = np.abs(x[i]) + np.abs(v[i] * dt) + np.abs(a[i]) * dt * dt + np.abs(j[i]) * dt ** 3
        assert np.all(np.abs(xp[i] - xo) <= 8 * 2.0 ** -53 * scale)
        assert np.all(np.abs(vp[i] - vo) <= 8 * 2.0 ** -53 * (np.abs(v[i]) + np.abs(a[i]) * dt + np.abs(j[i]) * dt * dt))


@pytest.mark.parametrize("n", [1, 31, 128, 129, 4097, 300001])
@pytest.mark.parametrize("pattern", ["random", "all", "first", "last", "sparse"])
def test_active_list_bit_exact(n, pattern):
    """The compaction's list as it sits in device memory (gd_active copies it
    out unchanged) equals the oracle's ascending list element by element, with
    the same block time; at n = 300001 the select grid's CTAs own several
    chunks each and a ragged last one."""
    rng = np.random.default_rng(n)
    m, x, v = inputs.plummer(n, seed=2)
    a = np.zeros((n, 3))
    jk = np.zeros((n, 3))
    if pattern == "all":
        dtau = np.full(n, 256, np.int64)
        tau = np.zeros(n, np.int64)
    else:
        dtau = 2 ** rng.integers(3, 9, size=n).astype(np.int64)
        tau = rng.integers(1, 6, size=n).astype(np.int64) * 256
        if pattern == "first":
            tau[:] = 2048
            dtau[:] = 256
            tau[0] = 1792
        elif pattern == "last":
            tau[:] = 2048
            dtau[:] = 256
            tau[-1] = 1792
        elif pattern == "sparse":
            tau[:] = 2048
            dtau[:] = 256
            pick = rng.choice(n, size=max(1, n // 1000), replace=False)
            tau[pick] = 1792
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        g.set_state(x, v, a, jk, tau, dtau)
        idx, tick = g.active()
    want, wt = oracle.active(tau + dtau)
    assert tick == wt
    assert np.array_equal(idx, want)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_matches_oracle(prec):
    """FP64 path: FP64 pairs.  Mixed path: FP32 pairs on double-single
    positions with a compensated sum; every term m_j / s_ij then carries at most
    about 8 units of 2^-24 (difference 2, r^2 3, refined rsqrt 2, product 1) and
    all terms have one sign, so |dU/U| <= 8 * 2^-24."""
    m, x, v = inputs.plummer(3001, seed=4)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec) as g:
        K, U = g.energy()
    Ko, Uo = oracle.energy(m, x, v, EPS)
    print("%s energy: dK/K %.2e dU/U %.2e" % (prec, K / Ko - 1, U / Uo - 1))
    assert K == pytest.approx(Ko, rel=1e-13)
    assert U == pytest.approx(Uo, rel=1e-12 if prec == "fp64" else 8 * U32)


def test_initial_state_matches_oracle():
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    so = sim.state()
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        st = g.state()
    np.testing.assert_allclose(st["a"], so["a"], rtol=0, atol=1e-12 * np.abs(so["a"]).max())
    np.testing.assert_allclose(st["j"], so["j"], rtol=0, atol=1e-12 * np.abs(so["j"]).max())
    assert (st["tau"] == 0).all()
    assert np.mean(st["dtau"] == so["dtau"]) > 0.99


def _replay(prec, m, x, v, rec):
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec) as g:
        E0 = sum(g.energy())
        for tick, idx in rec:
            g.replay_step(tick, idx)
        st = g.state()
        E1 = sum(g.energy())
        stats = g.stats()
    return st, E0, E1, stats


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_replayed_schedule_n512_to_t1(prec):
    """Plummer N = 512, eps = 1e-4, eta = 0.01, t = 0 -> 1, the GPU following
    the oracle's block schedule step by step."""
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    K0, U0 = sim.energy()
    rec = []
    while True:
        tick, idx = sim.step()
        rec.append((tick, idx))
        if tick >= int(1.0 / DT_MIN):
            break
    so = sim.state()
    K1, U1 = sim.energy()
    st, E0, E1, stats = _replay(prec, m, x, v, rec)
    assert stats["block_steps"] == len(rec)
    assert stats["particle_steps"] == sum(len(r[1]) for r in rec)
    de_or = (K1 + U1 - K0 - U0) / (K0 + U0)
    de_gpu = (E1 - E0) / E0
    dx = np.abs(st["x"] - so["x"]).max()
    agree = np.mean(st["dtau"] == so["dtau"])
    print("%s replay n=512: %d steps |dE/E| oracle %.3e gpu %.3e  max|dx| %.2e  dtau agree %.4f"
          % (prec, len(rec), abs(de_or), abs(de_gpu), dx, agree))
    assert (st["tau"] == so["tau"]).all()
    if prec == "fp64":
        assert dx < 1e-9
        assert abs(de_gpu - de_or) < 1e-10
        assert agree > 0.99
    else:
        assert dx < 1e-4
        assert abs(de_gpu) < 2 * abs(de_or) + 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_free_running_energy_within_2x_of_oracle(prec):
    m, x, v = inputs.plummer(512, seed=1)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    K0, U0 = sim.energy()
    sim.evolve(1.0)
    K1, U1 = sim.energy()
    de_or = abs((K1 + U1 - K0 - U0) / (K0 + U0))
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec) as g:
        E0 = sum(g.energy())
        g.evolve(1.0)
        E1 = sum(g.energy())
        st = g.state()
        stats = g.stats()
    de = abs((E1 - E0) / E0)
    so = sim.stats()
    print("%s free n=512 t=1: |dE/E| oracle %.3e gpu %.3e  blocks %d/%d  psteps %d/%d"
          % (prec, de_or, de, stats["block_steps"], so["nblock"], stats["particle_steps"], so["nsteps"]))
    assert (st["tau"] == int(1.0 / DT_MIN)).all()
    assert de <= 2 * de_or + 1e-9
    assert 0.8 < stats["block_steps"] / so["nblock"] < 1.25


def test_fp64_free_run_follows_the_oracle_schedule_n1024_to_t2():
    """The FP64 GPU path free-running from the benchmark's N = 1024 sphere to
    t = 2 (eta = 0.01) takes the oracle's block schedule: the same block and
    particle step counts (a quantisation decision could flip only for a step
    estimate within rounding of a power of two; allowed: 0.2 %) and the same
    energy error to within 5 %."""
    m, x, v = inputs.plummer(1024, seed=1)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    E0 = sum(sim.energy())
    sim.evolve(2.0)
    de_or = abs((sum(sim.energy()) - E0) / E0)
    so = sim.stats()
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        G0 = sum(g.energy())
        g.evolve(2.0)
        de = abs((sum(g.energy()) - G0) / G0)
        st = g.stats()
    print("fp64 n=1024 t=2: blocks %d/%d psteps %d/%d |dE/E| %.4e/%.4e"
          % (st["block_steps"], so["nblock"], st["particle_steps"], so["nsteps"], de, de_or))
    assert abs(st["block_steps"] - so["nblock"]) <= 0.002 * so["nblock"]
    assert abs(st["particle_steps"] - so["nsteps"]) <= 0.002 * so["nsteps"]
    assert abs(de - de_or) <= 0.05 * de_or


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1000, 20000])
def test_graph_eager_and_fused_paths_identical(prec, n):
    """The fused cooperative kernel, the captured graph and eager launches take
    the same block steps with the same arithmetic: bit-identical states."""
    m, x, v = inputs.plummer(n, seed=8)
    t_end = 0.25 if n <= 1000 else 0.125
    out = []
    for opts in (dict(fused=True), dict(fused=False, use_graph=True, graph_steps=7),
                 dict(fused=False, use_graph=False)):
        with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, **opts) as g:
            g.evolve(t_end)
            st = g.state()
            st["stats"] = np.array([g.stats()[k] for k in ("tick", "block_steps", "particle_steps")])
            out.append(st)
    for other in out[1:]:
        for k in out[0]:
            assert np.array_equal(out[0][k], other[k]), k


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cluster", [False, True])
def test_warp_mode_sums_in_force_kernel_or_corrector_identical(prec, cluster):
    """Warp-mode plans sum their j-split partials either in the force kernel (the
    last CTA of each tile, tuning mode 1) or in the corrector (mode 2); both take
    the same canonical order, so a run with either table is bit-identical."""
    n = 3000
    m, x, v = inputs.plummer(n, seed=31)
    if prec == "fp64" and cluster:
        pytest.skip("the cluster path is mixed precision only")
    out = []
    for mode in (1, 2):
        with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, cluster=cluster) as g:
            g.set_tuning(10 ** 9, np.full(32, 12, np.int16), np.full(32, mode, np.int8))
            assert (g.tuning()[2] == mode).all()
            g.evolve(0.125)
            st = g.state()
            st["stats"] = np.array([g.stats()[k] for k in ("tick", "block_steps", "particle_steps")])
            out.append(st)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("n", [1000, 4097, 20000])
def test_cluster_small_steps_vs_full_gpu(n):
    """Small block steps inside one thread-block cluster (the default) against
    every step on the full GPU: the same scheme and arithmetic, the force sums
    taken in another order, so the runs agree to round-off growth."""
    m, x, v = inputs.plummer(n, seed=12)
    t_end = 0.125
    res = {}
    for cl in (True, False):
        with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", cluster=cl) as g:
            info = g.cluster_info()
            E0 = sum(g.energy())
            g.evolve(t_end)
            E1 = sum(g.energy())
            res[cl] = (info, g.state(), g.stats(), (E1 - E0) / E0)
    (info1, st1, s1, de1), (info0, st0, s0, de0) = res[True], res[False]
    print("n=%d cluster %s: blocks %d/%d psteps %d/%d dE/E %.3e/%.3e"
          % (n, info1, s1["block_steps"], s0["block_steps"], s1["particle_steps"], s0["particle_steps"], de1, de0))
    assert info0[0] == 0
    assert info1[0] in (8, 16) and info1[1] * info1[0] >= n and 16 <= info1[2] <= 128
    tick = int(t_end / DT_MIN)
    assert (st1["tau"] == tick).all() and (st0["tau"] == tick).all()
    assert np.mean(st1["dtau"] == st0["dtau"]) > 0.99
    assert np.abs(st1["x"] - st0["x"]).max() < 1e-6
    assert abs(s1["particle_steps"] - s0["particle_steps"]) <= 0.01 * s0["particle_steps"]
    assert abs(de1) <= 2 * abs(de0) + 1e-9


def test_cluster_unsoftened_and_sizes():
    """eps = 0 (the unsoftened kernel instance) through the cluster path, and
    the sizes at which the cluster is not used."""
    m, x, v = inputs.plummer(500, seed=13)
    out = {}
    for cl in (True, False):
        with gravidy.Integrator(m, x, v, 0.0, ETA, precision="mixed", cluster=cl) as g:
            assert (g.cluster_info()[0] in (8, 16)) == cl
            E0 = sum(g.energy())
            g.evolve(0.125)  # dt_max: every particle's step divides it
            out[cl] = (g.state(), (sum(g.energy()) - E0) / E0)
    for cl, (st, de) in out.items():
        assert (st["tau"] == int(0.125 / DT_MIN)).all()
        assert np.isfinite(st["x"]).all() and np.isfinite(st["v"]).all()
    assert abs(out[True][1]) <= 2 * abs(out[False][1]) + 1e-9
    m, x, v = inputs.plummer(30000, seed=13)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        assert g.cluster_info() == (0, 0, 0)
    m, x, v = inputs.plummer(300, seed=13)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        assert g.cluster_info()[0] == 0


def test_step_block_matches_oracle_schedule():
    m, x, v = inputs.plummer(700, seed=9)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        for _ in range(50):
            tick, idx = sim.step()
            t, nact = g.step_block()
            assert t == tick * DT_MIN
            assert nact == idx.size


def test_checkpoint_restart_is_exact():
    m, x, v = inputs.plummer(900, seed=10)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        g.evolve(0.125)
        ck = {k: a.copy() for k, a in g.state().items()}
        g.evolve(0.25)
        ref = g.state()
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed") as g:
        g.set_state(ck["x"], ck["v"], ck["a"], ck["j"], ck["tau"], ck["dtau"])
        g.evolve(0.25)
        got = g.state()
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


def test_replay_rejects_a_particle_not_behind_the_block_time():
    m, x, v = inputs.plummer(64, seed=1)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision="fp64") as g:
        with pytest.raises(gravidy.GravidyError) as e:
            g.replay_step(0 + 1, [0, 1])          # fine: tau = 0 < 1
            g.replay_step(1, [0])                 # particle 0 is already at tick 1
        assert e.value.code == gravidy.GD_EINVAL


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("cluster", [False, True])
def test_kernel_timing_hook(fused, cluster):
    m, x, v = inputs.plummer(2000, seed=2)
    with gravidy.Integrator(m, x, v, EPS, ETA, time_force=True, fused=fused, cluster=cluster) as g:
        g.evolve(0.125)
        ms, launches, inter = g.kernel_time()
        cms, claunch = g.cluster_time()
        st = g.stats()
    total = st["interactions"] - 2000.0 ** 2   # all but the initial evaluation
    if fused:
        # the fused path times whole launches (cluster cycles included)
        assert 1 <= launches <= st["block_steps"]
        assert inter == total
    elif not cluster:
        assert launches == st["block_steps"] and inter == total and claunch == 0
    else:
        # the full-GPU force launches take the large steps, the cluster the rest
        assert 1 <= launches < st["block_steps"] and 0 < inter < total
        assert claunch >= 1 and cms > 0
    assert ms > 0
