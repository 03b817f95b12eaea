"""Two-body Kepler orbit in closed form (test helper, no oracle code).

A pair of equal masses m = 1/2 (total M = 1, G = 1) starts at pericentre of a
relative orbit with semi-major axis a and eccentricity e; kepler_at gives the
relative position and velocity at time t from Kepler's equation.
"""
import math

import numpy as np


def kepler_ic(e=0.5, a=1.0):
    m = np.array([0.5, 0.5])
    rp = a * (1 - e)
    vp = math.sqrt((1 + e) / (a * (1 - e)))
    x = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    v = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    return m, x, v


def kepler_at(t, e=0.5, a=1.0):
    """Relative position and velocity of a Kepler orbit (M = 1) that is at
    pericentre at t = 0, from Kepler's equation."""
    n = math.sqrt(1.0 / a ** 3)
    M = n * t
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    den = 1 - e * math.cos(E)
    r = np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    v = np.array([-a * n * math.sin(E) / den, a * n * math.sqrt(1 - e * e) * math.cos(E) / den, 0.0])
    return r, v
