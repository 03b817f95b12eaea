"""bench.py on the CPU: the reference arm (the oracle) prints one JSON line with
the fields the benchmark contract names, and the workload description matches
the GPU arm's."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "512",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["n"] == 512 and "plummer_n512" in d["config"]["workload"]


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_lagrange_radii_of_a_plummer_sphere_match_the_model():
    """Plummer model, scale length a: the mass inside r is r^3 / (r^2 + a^2)^(3/2),
    so the radius enclosing the fraction f is a / sqrt(f^(-2/3) - 1); in N-body
    units a = 3 pi / 16.  A 16384-particle sample about its density centre
    follows it to sampling noise."""
    import math

    import numpy as np

    from paper_1702_00440_gb300 import inputs
    bench = _bench()
    m, x, _ = inputs.plummer(16384, seed=5)
    a = 3 * math.pi / 16
    fr = [0.05, 0.1, 0.25, 0.5, 0.75]
    got = bench.lagrange_radii(m, x, fr, np.zeros(3))
    for f, r in zip(fr, got):
        want = a / math.sqrt(f ** (-2.0 / 3.0) - 1)
        assert abs(r / want - 1) < 0.05, (f, r, want)


def test_density_centre_finds_a_displaced_core():
    """A Plummer sphere shifted by c, plus a uniform halo of light particles that
    moves the centre of mass elsewhere: the density centre stays at c."""
    import numpy as np

    from paper_1702_00440_gb300 import inputs
    bench = _bench()
    m, x, _ = inputs.plummer(2048, seed=6)
    c = np.array([0.7, -0.3, 0.2])
    rng = np.random.default_rng(6)
    halo = rng.uniform(-20, -10, size=(512, 3))
    mm = np.concatenate([m, np.full(512, m[0])])
    xx = np.concatenate([x + c, halo])
    com = (mm[:, None] * xx).sum(0) / mm.sum()
    dc = bench.density_centre(mm, xx)
    assert np.linalg.norm(com - c) > 1.0
    assert np.linalg.norm(dc - c) < 0.05


def test_half_mass_relaxation_time_formula():
    """t_rh = 0.138 (N r_h^3 / <m>)^(1/2) / ln(0.1 N) for a sphere whose half-mass
    radius is known: a shell of unit radius (points in antipodal pairs, so its
    centre of mass is the origin) holds all its mass at r = 1."""
    import math

    import numpy as np
    bench = _bench()
    n = 4096
    rng = np.random.default_rng(7)
    u = rng.normal(size=(n // 2, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    x = np.concatenate([u, -u])
    m = np.full(n, 1.0 / n)
    trh, rh = bench.half_mass_relaxation_time(m, x)
    assert abs(rh - 1.0) < 1e-12
    assert abs(trh - 0.138 * math.sqrt(n * n) / math.log(0.1 * n)) < 1e-9 * trh


def test_collapse_sweep_oracle_leg_one_row():
    """The collapse sweep's oracle leg to 0.2 t_rh (one output at t = 4): the
    rows carry the diagnostics, the energy error is small and the block steps
    count up."""
    bench = _bench()
    res = bench._oracle_collapse_job((2, 0.2, 600.0))
    assert res["impl"] == "oracle" and res["seed"] == 2 and abs(res["t_rh"] - 20.18) < 0.01
    rows = res["rows"]
    assert [r["t"] for r in rows] == [0.0, 4.0]
    assert len(rows[1]["radii"]) == len(bench.COLLAPSE_FRACTIONS)
    assert all(a < b for a, b in zip(rows[1]["radii"], rows[1]["radii"][1:]))
    assert 0 < rows[1]["dE_E"] < 1e-6 and rows[1]["block_steps"] > 1000
