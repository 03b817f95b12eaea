"""High-precision pins of the oracle's force, jerk and snap on tiny systems.

Nothing here retypes the oracle's pair formulas.  At 40 significant digits
(mpmath), the acceleration of particle i is minus the gradient of the softened
potential Phi(y) = -sum_{j != i} m_j / sqrt(|x_j - y|^2 + eps^2) at y = x_i
(Eq. 1 as the gradient of the potential of Eq. 2, softened); the jerk is the
time derivative of that acceleration when every particle moves as x + v t; the
snap is its second time derivative when every particle moves as
x + v t + a t^2 / 2 (the sixth-order scheme's definition, with the particles'
accelerations a given).  The FP64 oracle must agree to round-off.
"""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from paper_1702_00440_gb300 import inputs  # noqa: E402

mp.mp.dps = 40


def _acc_mp(m, pos, i, eps2):
    """-grad Phi at particle i, for positions pos(j) (callables of nothing: mp values)."""
    def phi(y0, y1, y2):
        s = mp.mpf(0)
        for j in range(len(m)):
            if j == i:
                continue
            d0, d1, d2 = pos[j][0] - y0, pos[j][1] - y1, pos[j][2] - y2
            s -= mp.mpf(m[j]) / mp.sqrt(d0 * d0 + d1 * d1 + d2 * d2 + eps2)
        return s
    y = pos[i]
    return [-mp.diff(phi, (y[0], y[1], y[2]), tuple(1 if q == c else 0 for q in range(3))) for c in range(3)]


def _moving(x, v, b, t):
    return [[mp.mpf(x[j][c]) + mp.mpf(v[j][c]) * t + mp.mpf(b[j][c]) * t * t / 2 for c in range(3)]
            for j in range(len(x))]


def _system(n, seed, eps):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5, 2.0, n) / n
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3)) * 0.5
    return m, x, v, mp.mpf(eps) ** 2


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_force_and_jerk_against_the_potential_gradient(eps, oracle_mod):
    n = 7
    m, x, v, eps2 = _system(n, 31, eps)
    zero = np.zeros((n, 3))
    a_or, j_or = oracle_mod.force(m, x, v, eps)
    for i in range(n):
        a_mp = _acc_mp(m, _moving(x, v, zero, mp.mpf(0)), i, eps2)
        j_mp = [mp.diff(lambda t, c=c: _acc_mp(m, _moving(x, v, zero, t), i, eps2)[c], 0) for c in range(3)]
        for c in range(3):
            assert abs(a_or[i, c] - float(a_mp[c])) <= 1e-14 * max(1.0, abs(a_or[i]).max())
            assert abs(j_or[i, c] - float(j_mp[c])) <= 1e-13 * max(1.0, abs(j_or[i]).max())


def test_snap_against_the_second_time_derivative(oracle_mod):
    n = 6
    m, x, v, eps2 = _system(n, 32, 0.05)
    b = np.random.default_rng(33).normal(size=(n, 3))   # the particles' accelerations
    _, _, s_or = oracle_mod.force6(m, x, v, b, 0.05)
    for i in range(n):
        for c in range(3):
            s_mp = mp.diff(lambda t: _acc_mp(m, _moving(x, v, b, t), i, eps2)[c], 0, 2)
            assert abs(s_or[i, c] - float(s_mp)) <= 1e-12 * max(1.0, abs(s_or[i]).max())


def test_plummer_subset_force_to_round_off(oracle_mod):
    """Twelve particles of a Plummer sphere (close pairs included), eps = 1e-4:
    the relative error of the FP64 acceleration is at the round-off level."""
    m, x, v = inputs.plummer(12, seed=34)
    a_or, _ = oracle_mod.force(m, x, v, 1e-4)
    pos = _moving(x, v, np.zeros_like(x), mp.mpf(0))
    for i in range(12):
        a_mp = np.array([float(q) for q in _acc_mp(m, pos, i, mp.mpf(1e-4) ** 2)])
        assert np.linalg.norm(a_or[i] - a_mp) <= 1e-14 * np.linalg.norm(a_mp) * 12
