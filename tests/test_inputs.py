"""Pins of the seeded input generators (paper_1702_00440_gb300/inputs.py)
against the distributions they sample: the Plummer model's mass, centre,
truncation, energy and virial ratio in N-body units, its speed distribution
(q = v / v_esc with density q^2 (1 - q^2)^(7/2), whose mean of q^2 is
B(5/2, 9/2) / B(3/2, 9/2) = 1/4), isotropy; the power-law mass function's
range and quantiles; the log-uniform cluster sizes; the random subsets; and
reproducibility by seed."""
import math

import numpy as np
import pytest

from paper_1702_00440_gb300 import inputs

A = inputs.LENGTH_SCALE   # Plummer radius in N-body units, 3 pi / 16


@pytest.fixture(scope="module")
def big():
    return inputs.plummer(16384, seed=21)


def test_plummer_mass_centre_and_truncation(big):
    m, x, v = big
    assert abs(m.sum() - 1) < 1e-12 and np.all(m == m[0])
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-14
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-14
    # radii beyond 10 Plummer radii are redrawn (the centre-of-mass shift is tiny)
    assert np.linalg.norm(x, axis=1).max() < 10.0 * A * 1.001


def _truncated_plummer_energies(R=10.0):
    """K and U of the Plummer model cut at R Plummer radii with the mass beyond
    redrawn inside (density renormalised by M(R)), the speeds at each radius
    from the full model (<v^2> = (1/2) (1 + r^2)^(-1/2)), in G = M = a = 1 units,
    then in N-body units (lengths x 3 pi / 16, energies x 16 / (3 pi)).  Without
    the cut: K = 3 pi / 64, U = -3 pi / 32."""
    from scipy.integrate import quad
    M = lambda r: r ** 3 * (1 + r * r) ** -1.5
    dM = lambda r: 3 * r * r * (1 + r * r) ** -2.5
    MR = M(R)
    U = -quad(lambda r: M(r) * dM(r) / r, 0, R, limit=200)[0] / MR ** 2
    K = quad(lambda r: dM(r) * 0.25 * (1 + r * r) ** -0.5, 0, R, limit=200)[0] / MR
    s = 16 / (3 * math.pi)
    return K * s, U * s


def test_truncated_model_energies_reduce_to_the_plummer_closed_form():
    K, U = _truncated_plummer_energies(R=1e4)
    assert abs(K - 0.25) < 1e-6 and abs(U + 0.5) < 1e-4


def test_plummer_energy_and_virial_ratio():
    """A 4096-particle sample's kinetic and potential energy against the
    truncated model's (K = 0.2533, U = -0.5134, E = -0.2601 in N-body units: the
    1.5 % of the model's mass beyond 10 a, redrawn inside, binds it more than the
    untruncated E = -1/4); U of N particles carries the factor (1 - 1/N)."""
    Kt, Ut = _truncated_plummer_energies()
    m, x, v = inputs.plummer(4096, seed=22)
    K = 0.5 * (m * (v * v).sum(1)).sum()
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    iu = np.triu_indices(len(m), 1)
    U = -(m[iu[0]] * m[iu[1]] / d[iu]).sum()
    assert abs(K / Kt - 1) < 0.03
    assert abs(U / (Ut * (1 - 1 / len(m))) - 1) < 0.015


def test_plummer_speed_distribution(big):
    """q = |v| / v_esc(r) with v_esc = sqrt(2) (1 + r^2 / a^2)^(-1/4) / sqrt(a) in
    N-body units: mean q^2 = 1/4, and q < 1 (bound) for every particle up to the
    centre-of-mass correction."""
    m, x, v = big
    r = np.linalg.norm(x, axis=1)
    vesc = math.sqrt(2.0) * (1.0 + (r / A) ** 2) ** -0.25 / math.sqrt(A)
    q = np.linalg.norm(v, axis=1) / vesc
    assert abs((q * q).mean() - 0.25) < 0.006
    assert q.max() < 1.02


def test_plummer_isotropy(big):
    m, x, v = big
    s = (v * v).mean(0)
    assert np.abs(s / s.mean() - 1).max() < 0.03
    rhat = x / np.linalg.norm(x, axis=1)[:, None]
    vr2 = ((v * rhat).sum(1) ** 2).mean()
    vt2 = (v * v).sum(1).mean() - vr2
    assert abs(vt2 / (2 * vr2) - 1) < 0.05
    assert np.abs(rhat.mean(0)).max() < 0.03


def test_power_law_masses():
    """dN/dm ~ m^-2.35 on [0.2, 20], cumulative F(m) = (m_lo^-1.35 - m^-1.35) /
    (m_lo^-1.35 - m_hi^-1.35): the masses span at most a factor 100; F(x m_lo) =
    1/2 at x = 1.669 (the median over the smallest mass, which is m_lo to sampling
    precision); the fraction below 2 m_lo is (1 - 2^-1.35) / (1 - 100^-1.35) = 0.609."""
    m = inputs.power_law_masses(16384, seed=23)
    assert abs(m.sum() - 1) < 1e-12
    ratio = m / m.min()
    assert ratio.max() <= 100.0 * (1 + 1e-12)
    x_med = (1 - 0.5 * (1 - 100.0 ** -1.35)) ** (-1 / 1.35)
    assert abs(np.median(ratio) / x_med - 1) < 0.03
    f2 = (1 - 2.0 ** -1.35) / (1 - 100.0 ** -1.35)
    assert abs((ratio < 2).mean() - f2) < 0.015
    # the positions do not depend on the masses
    _, x1, _ = inputs.plummer(64, seed=5)
    _, x2, _ = inputs.plummer(64, seed=5, masses=inputs.power_law_masses(64, seed=5))
    shift = x2 - x1                    # the same sample up to the centre-of-mass shift
    assert np.ptp(shift, axis=0).max() < 1e-12


def test_ensemble_sizes_log_uniform():
    n = inputs.ensemble_sizes(256, seed=1)
    assert n.min() >= 256 and n.max() <= 8192 and n.dtype == np.int64
    ln = np.log(n + 0.5)
    mid = 0.5 * (math.log(256) + math.log(8192))
    assert abs(ln.mean() - mid) < 0.25
    assert np.array_equal(n, inputs.ensemble_sizes(256, seed=1))


def test_random_subset():
    idx = inputs.random_subset(1000, 137, seed=4)
    assert idx.dtype == np.int32 and len(idx) == 137 and len(np.unique(idx)) == 137
    assert np.all(np.diff(idx) > 0) and idx.min() >= 0 and idx.max() < 1000
    assert np.array_equal(idx, inputs.random_subset(1000, 137, seed=4))
    assert not np.array_equal(idx, inputs.random_subset(1000, 137, seed=5))
    assert np.array_equal(inputs.random_subset(10, 10, seed=1), np.arange(10))


def test_seeded_reproducibility():
    a = inputs.plummer(100, seed=7)
    b = inputs.plummer(100, seed=7)
    c = inputs.plummer(100, seed=8)
    for p, q in zip(a, b):
        assert np.array_equal(p, q)
    assert not np.array_equal(a[1], c[1])
    with pytest.raises(ValueError):
        inputs.plummer(0)
