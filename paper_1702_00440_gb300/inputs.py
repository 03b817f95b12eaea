"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.  This module holds sampling only -- none of the
integrator's arithmetic (no forces, energies, steps).

Plummer sphere: the sampling recipe of Aarseth, Henon & Wielen (1974), the
model GraviDy's tests use (Sec. 3.1: equal-mass Plummer spheres in standard
N-body units, G = M = 1, E = -1/4, Plummer radius about 0.6).  The model is
sampled in Plummer units (G = M = a = 1), the centre of mass is moved to the
origin at rest, and the sample is scaled to N-body units with the analytic
Plummer energy E = -3 pi / 64 (G M^2 / a): lengths multiplied by 3 pi / 16
and velocities by sqrt(16 / (3 pi)).  Radii beyond 10 Plummer radii are
redrawn; the model holds 1.5 % of its mass there, so the sample is a slightly
more bound, truncated model (K = 0.253, U = -0.513, E = -0.260 in these units)
plus a sampling fluctuation of order 1/sqrt(N); the paper's own initial
conditions were not exactly at -1/4 either (its log starts from E = -0.256,
Appendix A).

Power-law masses: dN/dm proportional to m^-2.35 on [0.2, 20] by inverse
transform sampling, rescaled so the masses sum to 1.
"""
from __future__ import annotations

import numpy as np

LENGTH_SCALE = 3.0 * np.pi / 16.0  # Plummer radius in N-body units


def _isotropic(rng, r):
    """Points of radius ``r`` with isotropic random directions."""
    n = r.shape[0]
    z = (1.0 - 2.0 * rng.random(n)) * r
    phi = 2.0 * np.pi * rng.random(n)
    rho = np.sqrt(np.maximum(r * r - z * z, 0.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def plummer(n: int, seed: int = 1, masses=None, rmax: float = 10.0):
    """Plummer sphere of ``n`` particles -> (m, x, v), float64, x/v shape (n, 3).

    ``masses`` None gives equal masses 1/n; otherwise an array of n masses that
    is rescaled to sum to 1.  Radii beyond ``rmax`` Plummer radii are redrawn.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    # radius from the inverse cumulative mass profile M(r) = r^3 / (1 + r^2)^(3/2)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        u = rng.random(todo.size)
        rr = np.where(u > 0, 1.0 / np.sqrt(np.maximum(u, 1e-300) ** (-2.0 / 3.0) - 1.0 + 1e-300), 0.0)
        ok = (u > 0) & (rr <= rmax)
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x = _isotropic(rng, r)
    # speed q * v_esc, v_esc = sqrt(2) (1 + r^2)^(-1/4); q from von Neumann
    # rejection on g(q) = q^2 (1 - q^2)^(7/2), whose maximum is below 0.1
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = rng.random(todo.size)
        x2 = rng.random(todo.size)
        ok = 0.1 * x2 < x1 * x1 * (1.0 - x1 * x1) ** 3.5
        q[todo[ok]] = x1[ok]
        todo = todo[~ok]
    speed = q * np.sqrt(2.0) * (1.0 + r * r) ** -0.25
    v = _isotropic(rng, speed)
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        if m.shape != (n,):
            raise ValueError("masses must have shape (n,)")
        m /= m.sum()
    # centre of mass at the origin, at rest
    mt = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt
    x *= LENGTH_SCALE
    v /= np.sqrt(LENGTH_SCALE)
    return m, np.ascontiguousarray(x), np.ascontiguousarray(v)


def power_law_masses(n: int, seed: int = 1, alpha: float = 2.35, m_lo: float = 0.2, m_hi: float = 20.0):
    """n masses with dN/dm ~ m^-alpha on [m_lo, m_hi], rescaled to sum to 1."""
    rng = np.random.default_rng(seed + 7919)
    u = rng.random(n)
    p = 1.0 - alpha
    m = (m_lo ** p + u * (m_hi ** p - m_lo ** p)) ** (1.0 / p)
    return m / m.sum()


def ensemble_sizes(nclusters: int = 256, seed: int = 1, n_lo: int = 256, n_hi: int = 8192):
    """Cluster sizes drawn log-uniformly from [n_lo, n_hi]."""
    rng = np.random.default_rng(seed + 104729)
    ln = rng.uniform(np.log(n_lo), np.log(n_hi), nclusters)
    return np.floor(np.exp(ln)).astype(np.int64)


def random_subset(n: int, k: int, seed: int = 1):
    """k distinct indices of range(n), ascending."""
    rng = np.random.default_rng(seed + 15485863)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
