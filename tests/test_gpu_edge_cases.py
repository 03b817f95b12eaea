"""Degenerate systems through the GPU integrator: a Kepler binary (N = 2,
unsoftened), an isolated particle (N = 1) and three bodies, in both precisions,
against closed forms and against the FP64 oracle.

With N <= 3 the mixed path runs every step inside the 16-CTA cluster kernel, so
the CTAs that own no particle take part in every barrier with empty loops.
"""
import numpy as np
import pytest

import oracle
from kepler import kepler_at, kepler_ic
from paper_1702_00440_gb300 import gravidy

pytestmark = pytest.mark.gpu

DT_MIN = 2.0 ** -22
ETA = 0.01


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gravidy.load()
    oracle.build()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_kepler_binary_matches_closed_form_and_oracle(prec):
    """e = 0.5 orbit, eps = 0, eta = 0.01, one period: the phase error of the
    4th-order scheme at this eta is below 1e-4; energy and eccentricity hold to
    1e-6 (FP64; 1e-5 mixed, whose forces carry FP32 rounding); the FP64 path
    follows the oracle's block schedule and state to round-off."""
    e, t_end = 0.5, 6.25
    m, x, v = kepler_ic(e)
    with gravidy.Integrator(m, x, v, 0.0, ETA, precision=prec) as g:
        if prec == "mixed":
            assert g.cluster_info()[0] in (8, 16)
        K0, U0 = g.energy()
        assert K0 + U0 == pytest.approx(-0.125, rel=1e-12)   # -m1 m2 / (2a)
        g.evolve(t_end)
        st = g.state()
        K, U = g.energy()
        stats = g.stats()
    assert (st["tau"] == int(t_end / DT_MIN)).all()
    r = st["x"][1] - st["x"][0]
    w = st["v"][1] - st["v"][0]
    r_ex, w_ex = kepler_at(t_end, e)
    tol = 1e-6 if prec == "fp64" else 1e-5
    print("%s kepler: |dr| %.2e |dw| %.2e dE/E %.2e blocks %d" % (prec, np.abs(r - r_ex).max(), np.abs(w - w_ex).max(),
                                                                (K + U) / (K0 + U0) - 1, stats["block_steps"]))
    assert np.abs(r - r_ex).max() < 1e-4
    assert np.abs(w - w_ex).max() < 1e-4
    assert abs((K + U) / (K0 + U0) - 1) < tol
    L = np.cross(r, w)
    ecc = np.cross(w, L) - r / np.linalg.norm(r)
    assert abs(np.linalg.norm(ecc) - e) < tol
    # the centre of mass stays at rest (both bodies always share the block step)
    assert np.abs((m[:, None] * st["v"]).sum(0)).max() < 1e-12
    if prec == "fp64":
        sim = oracle.Sim(m, x, v, 0.0, ETA)
        sim.evolve(t_end)
        so = sim.state()
        assert stats["block_steps"] == sim.stats()["nblock"]
        assert np.abs(st["x"] - so["x"]).max() < 1e-10
        assert np.abs(st["v"] - so["v"]).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_isolated_particle_moves_uniformly(prec):
    """N = 1: no force, the step criterion is unconstrained (0/0), the step grows
    to dt_max, and the particle moves on a straight line; the energy is its
    kinetic energy."""
    m = np.array([1.0])
    x = np.array([[0.3, -0.2, 0.1]])
    v = np.array([[0.5, 0.25, -0.125]])
    with gravidy.Integrator(m, x, v, 1e-4, ETA, precision=prec) as g:
        g.evolve(1.0)
        st = g.state()
        K, U = g.energy()
    assert np.abs(st["x"] - (x + v)).max() < 1e-13
    assert np.abs(st["v"] - v).max() == 0.0
    assert np.abs(st["a"]).max() == 0.0 and np.abs(st["j"]).max() == 0.0
    assert st["dtau"][0] == int(0.125 / DT_MIN)
    assert K == pytest.approx(0.5 * np.dot(v[0], v[0]), rel=1e-14) and U == 0.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_bodies_against_the_oracle(prec):
    """A bound three-body system (eps = 1e-3) to t = 1: the FP64 path takes the
    oracle's schedule and state to round-off growth; the mixed path stays within
    the integrator's own error of it."""
    m = np.array([0.5, 0.3, 0.2])
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.1], [-0.6, 0.7, -0.2]])
    v = np.array([[0.0, -0.1, 0.0], [0.05, 0.6, 0.0], [-0.3, -0.2, 0.1]])
    cm = (m[:, None] * v).sum(0) / m.sum()
    v = v - cm
    sim = oracle.Sim(m, x, v, 1e-3, ETA)
    E0 = sum(sim.energy())
    sim.evolve(1.0)
    so = sim.state()
    de_or = abs((sum(sim.energy()) - E0) / E0)
    with gravidy.Integrator(m, x, v, 1e-3, ETA, precision=prec) as g:
        G0 = sum(g.energy())
        g.evolve(1.0)
        st = g.state()
        de = abs((sum(g.energy()) - G0) / G0)
    dx = np.abs(st["x"] - so["x"]).max()
    print("%s three bodies: |dx| vs oracle %.2e  |dE/E| %.2e (oracle %.2e)" % (prec, dx, de, de_or))
    if prec == "fp64":
        assert (st["dtau"] == so["dtau"]).all()
        assert dx < 1e-10
        assert abs(de - de_or) <= 1e-3 * de_or + 1e-14
    else:
        assert dx < 1e-5
        assert de <= 2 * de_or + 1e-9
