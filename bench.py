#!/usr/bin/env python
"""Benchmark of the GB300 Hermite-4 block-step N-body hot path.

Workload: Plummer sphere, N = 16384 equal masses in N-body units, Plummer
softening eps = 1e-4, Aarseth eta = 0.01, power-of-two block steps in
[2^-22, 1/8], mixed precision (FP32 pair arithmetic on double-single positions
with compensated FP32 sums; prediction, correction and the Aarseth step in
double-single / FP32 arithmetic; integer block-time bookkeeping; energy pair
terms in FP32 with compensated sums and FP64 totals).  One benchmark step advances the
system by dt_max = 1/8 N-body time unit -- every block step in that interval
(active-list compaction, prediction of all N, force/jerk of the active set with
j-split reduction, correction + Aarseth step + quantisation) -- and evaluates
the energy at the synchronised end time, i.e. one output row of GraviDy's run
log (Appendix A).  Metric: acc+jerk interactions per second (sum of N_act * N
over all force evaluations of the timed steps / device time).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "acc+jerk interactions/s (%FP32 peak @60 flop); s per N-body time unit at |dE/E|"
UNIT = "interactions/s"
N_DEFAULT = 16384
EPS = 1e-4
ETA = 0.01
DT_STEP = 0.125
FLOP_PER_INTERACTION = 60
# FP32 non-tensor peak from unit counts and the maximum SM clock:
# 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) of one launch per kernel, from one ncu --set full
# capture of the steady-state block steps of this workload (ncu's default cache
# control: caches flushed before the launch), keyed by the SHA-256 of the kernel
# sources the capture ran on; a changed source reports null.
TRAFFIC_PER_LAUNCH = {
    "481ff2b6": {"k_cluster_steps": 1570560, "k_force_mixed": 714880},
    # 481ff2b6 plus the failure-detection probe kernel, its host call and the
    # grid barrier's poll loop moved into a helper: the two captured kernels'
    # code is unchanged
    "ba8ae45d": {"k_cluster_steps": 1570560, "k_force_mixed": 714880},
    # asynchronous double-buffered j-tiles in the force kernel, per-bucket choice of
    # where warp-mode j-split sums are taken
    "2d1d3ec0": {"k_cluster_steps": 1582080, "k_force_mixed": 716288},
    # 2d1d3ec0 plus the 2PN pair terms (only in the corrector and the force hooks),
    # then plus the P(EC)^n trial passes of the corrector (a branch the captured force
    # kernel compiles out): the two captured kernels' memory accesses are unchanged
    "ddb7dccc": {"k_cluster_steps": 1582080, "k_force_mixed": 716288},
    "fe3ba5e9": {"k_cluster_steps": 1582080, "k_force_mixed": 716288},
    # j-loops unrolled 8 in the force kernel and the cluster's force tasks
    "2dc045bc": {"k_cluster_steps": 1579264, "k_force_mixed": 722688},
    # 2dc045bc plus the independent-cluster ensemble kernel (a separate file) and the
    # post-Newtonian pair in the cluster's correction (a branch the benchmark, with no
    # pair, does not take): the two captured kernels' memory accesses are unchanged
    "e180922f": {"k_cluster_steps": 1579264, "k_force_mixed": 722688},
    # e180922f with the cluster kernel's pair terms and P(EC)^n passes in a separate
    # template instance (the benchmark launches the plain one)
    "e618334d": {"k_cluster_steps": 1579264, "k_force_mixed": 722688},
    # e618334d with the cluster's partial forces at a padded slot stride (shared memory
    # only: the DRAM accesses are unchanged)
    "fdc36443": {"k_cluster_steps": 1579264, "k_force_mixed": 722688},
    # fdc36443 with host-side changes to the ensemble launches only: the captured
    # kernels are unchanged
    "5fc3df47": {"k_cluster_steps": 1579264, "k_force_mixed": 722688},
}


def _args():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gravidy", choices=["gravidy", "reference"])
    p.add_argument("--n", type=int, default=N_DEFAULT)
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-extras", action="store_true", help="skip the fp64, force-sweep, e2e and cpu legs")
    p.add_argument("--no-autotune", action="store_true", help="use the default force-kernel tuning table")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample length")
    p.add_argument("--sweep-n", type=int, default=1 << 20)
    p.add_argument("--profile-force", type=int, default=0, metavar="N",
                   help="profiling hook: initialise an N-particle Plummer sphere (one full force evaluation), "
                        "evaluate all N once more, print nothing and exit")
    p.add_argument("--sweep", choices=["force", "powerlaw", "accuracy", "ensemble", "eta", "soft", "lagrange", "h6",
                                          "timesym", "collapse", "fp32peak", "cluster"],
                   help="extra measurements, one JSON line each (not the benchmark line): force = "
                        "full evaluations N=2^10..2^20 and N=2^20 with active sets 1..2^20; powerlaw = "
                        "N=262144 power-law masses to t=1/8 (active-set histogram, interactions/s per "
                        "set size); accuracy = N=16384 FP64 vs mixed to t=1; ensemble = 256 clusters of "
                        "log-uniform N in [256, 8192] to t=--ens-t, one ensemble vs the clusters one by one; eta = "
                        "Plummer N=1024..16384 to t=2 for eta=0.001..0.1: s per N-body unit and |dE/E| (mixed, FP64 "
                        "at eta=0.01, the oracle at N=1024) and the block-step distribution; soft = the same for "
                        "eps=1e-5..1e-2 at eta=0.01; lagrange = Lagrange radii of N=16384 every 1/2 unit to t=8; "
                        "h6 = sixth- vs fourth-order Hermite: cost and |dE/E| to t=1, and the snap kernel's rate; "
                        "timesym = the time-symmetric schemes (order 4 and 6, one and two passes): cost and |dE/E| "
                        "to t=1, energy drift and reversibility on a Kepler orbit with shared constant steps; "
                        "collapse = core collapse of an N=1024 Plummer sphere (Lagrange radii, |dE/E|); "
                        "fp32peak = the FP32 FMA throughput probe (the force kernels' roofline denominator) with "
                        "the SM clock sampled during it; cluster = where the small-step cluster's time goes on "
                        "the --n workload over one N-body unit (phase cycle counters, per small step)")
    p.add_argument("--ens-t", type=float, default=0.125)
    p.add_argument("--collapse-trh", type=float, default=30.0,
                   help="--sweep collapse: stop at this many half-mass relaxation times")
    p.add_argument("--collapse-wall", type=float, default=240.0,
                   help="--sweep collapse: stop each run after this many seconds of wall time")
    p.add_argument("--collapse-seeds", default="1", help="--sweep collapse: comma-separated Plummer seeds")
    p.add_argument("--collapse-oracle", action="store_true",
                   help="--sweep collapse: run the FP64 oracle on the host cores (one seed per core) instead of "
                        "the GPU")
    p.add_argument("--profile-force-h6", type=int, default=0, metavar="N",
                   help="profiling hook: initialise an N-particle Plummer sphere on the sixth-order path (two "
                        "force/jerk/snap evaluations), evaluate all N once more, print nothing and exit")
    p.add_argument("--profile-nact", type=int, default=0, metavar="K",
                   help="profiling hook: autotune on the --n workload, then evaluate the force of K random "
                        "particles (gd_force) once, and twice more between cudaProfilerStart/Stop; print the "
                        "tuning table and exit")
    p.add_argument("--profile-ensemble", type=int, default=0, metavar="K",
                   help="profiling hook: the first K clusters of the 256-cluster ensemble workload, advanced "
                        "from t = 0 to 1/64 between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    p.add_argument("--profile-steps", type=int, default=0, metavar="K",
                   help="profiling hook: integrate the --n workload to t = 0.375, then advance K/64 "
                        "N-body time units between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return p.parse_args()


def _workload(n):
    return {
        "workload": "plummer_n%d_equal_mass_eps1e-4_eta0.01_blocksteps_2^-22..1/8" % n,
        "n": n,
        "eps": EPS,
        "eta": ETA,
        "dt_min": 2.0 ** -22,
        "dt_max": DT_STEP,
        "step": "advance 1/8 N-body time unit (all block steps) + energy at the synchronised end",
        "ics": "Aarseth-Henon-Wielen Plummer sampling, seed 1 (+rank), N-body units",
        "l2": "flushed between timed steps (512 MiB device write outside the events)",
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [q.strip() for q in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower().startswith("active")})
        sm = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows), "samples": len(rows),
                "reasons": reasons}


def _rejected(clocks):
    if not clocks:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clocks["reasons"]):
        return True
    return clocks["sm_mhz"] < 0.5 * clocks["sm_max_mhz"] and not clocks["reasons"]


# ------------------------------------------------------------------ distributed

def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class _Comm:
    def __init__(self, world, rank, use_cuda):
        self.world, self.rank = world, rank
        self.dist = None
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("nccl" if use_cuda else "gloo")
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def reduce(self, value, op):
        if not self.dist:
            return value
        import torch

        t = torch.tensor([float(value)], dtype=torch.float64,
                         device="cuda" if self.dist.get_backend() == "nccl" else "cpu")
        self.dist.all_reduce(t, op=getattr(self.dist.ReduceOp, op))
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


# ------------------------------------------------------------------ oracle legs

def _oracle_sample(n, seconds, seed=1):
    """Time the FP64 oracle integrator on the benchmark's initial conditions:
    its initial O(N^2) force plus as many block steps as fit in ``seconds``."""
    import oracle
    from paper_1702_00440_gb300 import inputs

    m, x, v = inputs.plummer(n, seed=seed)
    t0 = time.perf_counter()
    sim = oracle.Sim(m, x, v, EPS, ETA)
    steps = 0
    while time.perf_counter() - t0 < seconds:
        sim.step()
        steps += 1
    dt = time.perf_counter() - t0
    st = sim.stats()
    return st["interactions"] / dt, st, dt, steps


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1702_00440_gb300 import inputs

    oracle.build()
    n = a.n
    m, x, v = inputs.plummer(n, seed=1)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    per_step = 40  # oracle block steps per benchmark step

    def one():
        t0 = time.perf_counter()
        it0 = sim.stats()["interactions"]
        for _ in range(per_step):
            sim.step()
        return sim.stats()["interactions"] - it0, time.perf_counter() - t0

    for _ in range(a.warmup):
        one()
    tot_i = tot_t = 0.0
    for _ in range(a.steps):
        i, t = one()
        tot_i += i
        tot_t += t
    value = tot_i / tot_t
    sample = ("oracle block steps on the N=%d Plummer ICs after its initial force: %d timed steps of %d block "
              "steps each (%.3g interactions in %.2f s), single-threaded FP64 C" % (n, a.steps, per_step, tot_i, tot_t))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * tot_t / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _workload(n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ main arm

# the sources the fourth-order step kernels are built from (the sixth-order path,
# hermite6.cu, has kernels of its own)
STEP_SOURCES = ("cluster.cuh", "ensemble.cuh", "gravidy.cu", "kernels.cuh")


def _csrc_hash():
    """SHA-256 over the step kernels' CUDA sources (file names and contents)."""
    d = os.path.join(ROOT, "paper_1702_00440_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name in STEP_SOURCES:
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def _traffic(kernel):
    return TRAFFIC_PER_LAUNCH.get(_csrc_hash()[:8], {}).get(kernel)


def run_gravidy(a):
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    comm = _Comm(world, rank, True)
    gravidy.load()
    n = a.n
    stream = torch.cuda.Stream()
    m, x, v = inputs.plummer(n, seed=1 + rank)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)

    g = gravidy.Integrator(m, x, v, EPS, ETA, precision=a.precision, stream=stream.cuda_stream,
                           autotune=not a.no_autotune)
    K0, U0 = g.energy()
    E0 = K0 + U0
    t = 0.0
    for _ in range(a.warmup):
        t += DT_STEP
        g.evolve(t)
        g.energy()

    def timed_region():
        nonlocal t, start
        # the state at the start of the timed steps: the roofline and e2e passes below
        # replay exactly these block steps from it
        start = (t, {k: q.copy() for k, q in g.state().items()})
        s0 = g.stats()
        comm.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        total_ms = 0.0
        per = []
        E = None
        # cudaProfilerStart/Stop bracket the timed steps, so that a profiler run with
        # --profile-from-start off sees exactly them (no effect otherwise)
        torch.cuda.profiler.start()
        for _ in range(a.steps):
            flush_l2()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t += DT_STEP
            g.evolve(t)
            Kx, Ux = g.energy()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            per.append(ms)
            total_ms += ms
            E = Kx + Ux
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        comm.barrier()
        clocks = sampler.stop()
        s1 = g.stats()
        return total_ms, per, E, clocks, s0, s1

    start = None
    total_ms, per, E, clocks, s0, s1 = timed_region()
    retried = False
    if _rejected(clocks):
        retried = True
        total_ms, per, E, clocks, s0, s1 = timed_region()
    inter = s1["interactions"] - s0["interactions"]
    launches = s1["kernel_launches"] - s0["kernel_launches"]
    max_ms = comm.reduce(total_ms, "MAX")
    tot_inter = comm.reduce(inter, "SUM")
    value = tot_inter / (max_ms / 1e3)
    nbu = a.steps * DT_STEP
    de = abs((E - E0) / E0)
    t_w, st_w = start
    tuning = g.tuning()

    # ---- roofline of the force and cluster kernels: the timed block steps replayed
    # from their starting state, with the same tuning table (so the same block steps
    # and arithmetic) and CUDA events around every force and cluster launch
    g2 = gravidy.Integrator(m, x, v, EPS, ETA, precision=a.precision, stream=stream.cuda_stream, time_force=True)
    g2.set_tuning(*tuning[:3])
    g2.set_state(st_w["x"], st_w["v"], st_w["a"], st_w["j"], st_w["tau"], st_w["dtau"])
    g2.kernel_time()
    g2.cluster_time()
    s2a = g2.stats()
    t2 = t_w
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    region_ms = 0.0
    for _ in range(a.steps):
        flush_l2()
        e0.record(stream)
        t2 += DT_STEP
        g2.evolve(t2)
        g2.energy()
        e1.record(stream)
        e1.synchronize()
        region_ms += e0.elapsed_time(e1)
    f_ms, f_launches, f_inter = g2.kernel_time()
    c_ms, c_launches = g2.cluster_time()
    cl_size, _, cl_ns = g2.cluster_info()
    s2b = g2.stats()
    g2.close()
    same_steps = (s2b["block_steps"] - s2a["block_steps"] == s1["block_steps"] - s0["block_steps"]
                  and s2b["interactions"] - s2a["interactions"] == inter)
    # the block steps the cluster took: every interaction of the region outside
    # the full-GPU force launches
    c_inter = max(0.0, (s2b["interactions"] - s2a["interactions"]) - f_inter)
    peak_basis = "FP32 non-tensor: 152 SMs x 128 lanes x 2 flop x 2070 MHz (unit counts x max clock)"
    kernels = {}
    fname = "k_force_%s" % ("mixed" if a.precision == "mixed" else "fp64")
    for name, ms, nl, k_inter in ((fname, f_ms, f_launches, f_inter),
                                  ("k_cluster_steps", c_ms, c_launches, c_inter)):
        if nl <= 0 or ms <= 0:
            continue
        ach = FLOP_PER_INTERACTION * k_inter / (ms / 1e3) / 1e12
        kernels[name] = {
            "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS, "traffic": _traffic(name), "kernel": name,
            "peak_basis": peak_basis, "flop_per_interaction": FLOP_PER_INTERACTION, "launches": nl,
            "avg_launch_us": 1e3 * ms / nl, "interactions_per_launch": k_inter / nl,
            "share_of_step_time": ms / region_ms if region_ms > 0 else None,
        }
    if "k_cluster_steps" in kernels:
        # the cluster runs on cl_size SMs by design (small steps are latency bound)
        kc = kernels["k_cluster_steps"]
        kc["cluster_ctas"] = cl_size
        kc["max_nact_per_step"] = cl_ns
        kc["frac_of_cluster_sms"] = kc["frac"] * SMS / cl_size
        kc["block_steps_per_launch"] = (s2b["block_steps"] - s2a["block_steps"] - f_launches) / kc["launches"]
    # the roofline object is the kernel with the largest share of the step time
    dominant = max(kernels.values(), key=lambda q: q["share_of_step_time"] or 0.0)
    roofline = dict(dominant)
    roofline["other_kernels"] = {k: q for k, q in kernels.items() if k != dominant["kernel"]}

    extras = {}
    cpu = None
    e2e = None
    if not a.no_extras:
        # ---- end to end through the public API from pinned host buffers: the timed
        # block steps replayed from their starting state, every step's state uploaded
        # from and read back to pinned host memory
        pin = {k: torch.empty(q.shape, dtype=torch.float64 if q.dtype == np.float64 else torch.int64,
                              pin_memory=True).numpy() for k, q in st_w.items()}
        for k in pin:
            pin[k][...] = st_w[k]
        t_e = t_w
        bi = 4 * n * 3 * 8 + 3 * n * 8   # x, v, a, jerk + tau, dtau, next time
        bo = 4 * n * 3 * 8 + 2 * n * 8 + 16
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        e_inter = 0.0
        e_blocks = 0
        for _ in range(a.steps):
            s_i = g.stats()
            g.set_state(pin["x"], pin["v"], pin["a"], pin["j"], pin["tau"], pin["dtau"])
            t_e += DT_STEP
            g.evolve(t_e)
            g.energy()
            g.state(out=pin)
            s_o = g.stats()
            e_inter += s_o["interactions"] - s_i["interactions"]
            e_blocks += s_o["block_steps"] - s_i["block_steps"]
        w1 = time.perf_counter()
        e_max = comm.reduce(w1 - w0, "MAX")
        e2e = {"value": comm.reduce(e_inter, "SUM") / e_max, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "same_block_steps_as_value": e_inter == inter,
               "interactions": e_inter, "block_steps": e_blocks, "value_interactions": inter,
               "value_block_steps": s1["block_steps"] - s0["block_steps"],
               "timing": "host wall clock, set_state + evolve(+1/8) + energy + get_state, replaying the timed "
                         "block steps from their starting state"}

        # ---- plain FP64 GPU form over the first 1/8 from the same ICs
        if a.precision == "mixed":
            for prec in ("fp64", "mixed"):
                g3 = gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, stream=stream.cuda_stream)
                Ea = sum(g3.energy())
                e0.record(stream)
                g3.evolve(DT_STEP)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                Eb = sum(g3.energy())
                st3 = g3.stats()
                g3.close()
                extras["t0_to_1/8_%s" % prec] = {"s_per_nbu": ms / 1e3 / DT_STEP, "dE_E": abs((Eb - Ea) / Ea),
                                                 "interactions_per_s": (st3["interactions"] - n * n) / (ms / 1e3)}

        # ---- full force evaluation at N = 2^20 (all particles active)
        if rank == 0 and a.sweep_n > 0:
            ms_, xs_, vs_ = inputs.plummer(a.sweep_n, seed=1)
            g4 = gravidy.Integrator(ms_, xs_, vs_, EPS, ETA, precision="mixed", stream=stream.cuda_stream,
                                    time_force=True)
            g4.kernel_time()
            idx = np.arange(a.sweep_n, dtype=np.int32)
            g4.force(0, idx)
            g4.kernel_time()
            g4.force(0, idx)
            fm, fl, fi = g4.kernel_time()
            g4.close()
            extras["force_full_n%d" % a.sweep_n] = {
                "interactions_per_s": fi / (fm / 1e3), "ms": fm,
                "tflops_at_60": FLOP_PER_INTERACTION * fi / (fm / 1e3) / 1e12,
                "frac_fp32_peak": FLOP_PER_INTERACTION * fi / (fm / 1e3) / 1e12 / FP32_PEAK_TFLOPS}

        # ---- the oracle on the host cores (rank 0, single GPU only)
        if rank == 0 and world == 1:
            cv, cst, cdt, csteps = _oracle_sample(n, a.cpu_seconds)
            cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "FP64 C oracle on the same N=%d ICs: initial O(N^2) force + %d block steps "
                             "(%.3g interactions in %.1f s)" % (n, csteps, cst["interactions"], cdt)}
    g.close()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": max_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair / ds-f32 update" if a.precision == "mixed" else "f64",
            "data": "synthetic", "config": _workload(n),
            "s_per_nbu": max_ms / 1e3 / nbu, "dE_E": de,
            "t_timed": [t_w, t_w + a.steps * DT_STEP], "roofline_same_block_steps": same_steps,
            "block_steps": s1["block_steps"] - s0["block_steps"],
            "particle_steps": s1["particle_steps"] - s0["particle_steps"],
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "clock_retry": retried, "per_step_ms": per, **extras,
        }
        print(json.dumps(out))
    comm.close()
    return 0


def _timed_force(g, idx, reps=3):
    """Median force-kernel time (ms) of gd_force over idx, CUDA events."""
    ts = []
    g.kernel_time()
    for _ in range(reps):
        g.force(0, idx)
        ms, _, _ = g.kernel_time()
        ts.append(ms)
    return sorted(ts)[len(ts) // 2]


# ------------------------------------------------------------------ oracle on all host cores

def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _pool(workers):
    """A process pool started with spawn (the parent holds a CUDA context)."""
    import multiprocessing as mp

    return mp.get_context("spawn").Pool(workers)


def _oracle_cluster_job(job):
    """One cluster of the ensemble through the oracle to t_end: (interactions, s)."""
    q, n, seed, t_end = job
    import oracle
    from paper_1702_00440_gb300 import inputs

    m, x, v = inputs.plummer(int(n), seed=int(seed))
    t0 = time.perf_counter()
    sim = oracle.Sim(m, x, v, EPS, ETA)
    sim.evolve(t_end)
    return sim.stats()["interactions"], time.perf_counter() - t0


def _oracle_compare_job(job):
    """One ensemble cluster: the oracle's run to t and the energy errors of its
    state and of the GPU's state at t, both by the oracle's FP64 energy function:
    (cluster, interactions, s, |dE/E| GPU, |dE/E| oracle)."""
    q, n, seed, t_end, xg, vg = job
    import oracle
    from paper_1702_00440_gb300 import inputs

    m, x, v = inputs.plummer(int(n), seed=int(seed))
    E0 = sum(oracle.energy(m, x, v, EPS))
    Eg = sum(oracle.energy(m, xg, vg, EPS))
    t0 = time.perf_counter()
    sim = oracle.Sim(m, x, v, EPS, ETA)
    sim.evolve(t_end)
    wall = time.perf_counter() - t0
    Eo = sum(sim.energy())
    return q, sim.stats()["interactions"], wall, abs((Eg - E0) / E0), abs((Eo - E0) / E0)


def _oracle_force_job(job):
    """Oracle force of a slice of active particles against all n: (count, s)."""
    n, idx = job
    import oracle
    from paper_1702_00440_gb300 import inputs

    m, x, v = inputs.plummer(int(n), seed=1)
    t0 = time.perf_counter()
    oracle.force(m, x, v, EPS, np.asarray(idx, dtype=np.int32))
    return len(idx), time.perf_counter() - t0


def sweep_force(a):
    """Full evaluations N = 2^10..2^20 (mixed), and N = 2^20 with random active
    sets of 1, 32, 1024, 32768, 2^20 (mixed and FP64, FP64 up to 32768), with the
    oracle timed on a bounded i-subsample against all N."""
    import oracle
    from paper_1702_00440_gb300 import gravidy, inputs

    gravidy.load()
    rows = []
    for k in range(10, 21):
        n = 1 << k
        m, x, v = inputs.plummer(n, seed=1)
        with gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", time_force=True) as g:
            ms = _timed_force(g, np.arange(n, dtype=np.int32))
        ips = float(n) * n / (ms / 1e3)
        rows.append({"n": n, "nact": n, "precision": "mixed", "ms": ms, "interactions_per_s": ips,
                     "frac_fp32_peak": FLOP_PER_INTERACTION * ips / 1e12 / FP32_PEAK_TFLOPS})
    n = 1 << 20
    m, x, v = inputs.plummer(n, seed=1)
    for prec in ("mixed", "fp64"):
        with gravidy.Integrator(m, x, v, EPS, ETA, precision=prec, time_force=True, autotune=prec == "mixed") as g:
            for nact in (1, 32, 1024, 32768, n):
                if prec == "fp64" and nact > 32768:
                    continue
                idx = np.arange(n, dtype=np.int32) if nact == n else inputs.random_subset(n, nact, seed=nact)
                ms = _timed_force(g, idx)
                ips = float(nact) * n / (ms / 1e3)
                rows.append({"n": n, "nact": nact, "precision": prec, "ms": ms, "interactions_per_s": ips,
                             "frac_fp32_peak": FLOP_PER_INTERACTION * ips / 1e12 / FP32_PEAK_TFLOPS,
                             "j_bytes_per_s": 40.0 * n / (ms / 1e3)})
    oracle.build()
    sub = inputs.random_subset(n, 64, seed=4096)
    t0 = time.perf_counter()
    oracle.force(m, x, v, EPS, sub)
    dt = time.perf_counter() - t0
    # the 4096-particle i-subsample against all 2^20 j, spread over the host cores
    cores = _host_cores()
    sub4k = inputs.random_subset(n, 4096, seed=4096)
    jobs = [(n, part.tolist()) for part in np.array_split(sub4k, cores)]
    t0 = time.perf_counter()
    with _pool(cores) as pool:
        done = pool.map(_oracle_force_job, jobs)
    dt4k = time.perf_counter() - t0
    out = {"sweep": "force", "metric": "acc+jerk interactions/s", "rows": rows,
           "oracle": {"interactions_per_s": 64.0 * n / dt, "sample": "64 i x 2^20 j", "cores": 1},
           "oracle_all_cores": {"interactions_per_s": 4096.0 * n / dt4k, "wall_s": dt4k, "cores": cores,
                                "sample": "4096 i x 2^20 j (wall time includes each worker's start and its "
                                          "regeneration of the 2^20 inputs)",
                                "worker_s": [round(w, 2) for _, w in done]},
           "peak_tflops": FP32_PEAK_TFLOPS}
    print(json.dumps(out))
    return 0


def sweep_powerlaw(a):
    """N = 262144 Plummer with power-law masses, mixed, t = 0 -> 1/8: active-set
    size histogram per block step, the autotuner's force time per set-size bucket
    (interactions/s per block size), wall time per N-body unit and |dE/E|."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    n = 262144
    m, x, v = inputs.plummer(n, seed=3, masses=inputs.power_law_masses(n, seed=3))
    g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", autotune=True)
    mode_cut, split, mode, tms = g.tuning()
    K0, U0 = g.energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.evolve(DT_STEP)
    wall = time.perf_counter() - t0
    K1, U1 = g.energy()
    st = g.stats()
    g.close()
    # the same run on the cooperative fused path (every block step inside persistent
    # launches: no per-step kernel launches), with the same tuning table
    g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", fused=True)
    g.set_tuning(mode_cut, split, mode)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.evolve(DT_STEP)
    wall_f = time.perf_counter() - t0
    Kf, Uf = g.energy()
    stf = g.stats()
    g.close()
    fused = {"wall_s": wall_f, "s_per_nbu": wall_f / DT_STEP, "block_steps": stf["block_steps"],
             "particle_steps": stf["particle_steps"], "dE_E": abs((Kf + Uf - K0 - U0) / (K0 + U0))}
    # the same run again one block step at a time, for the active-set histogram
    g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed")
    hist = {}
    steps = 0
    while True:
        t, nact = g.step_block()
        steps += 1
        b = int(np.log2(nact))
        hist[b] = hist.get(b, 0) + 1
        if t >= DT_STEP:
            break
    g.close()
    per_bucket = []
    for b in sorted(hist):
        row = {"log2_nact": b, "block_steps": hist[b]}
        if tms[b] > 0:
            row["force_ms"] = float(tms[b])
            row["interactions_per_s"] = float(2 ** b) * n / (float(tms[b]) / 1e3)
            row["mode"] = {0: "i-parallel", 1: "warp", 2: "warp, sums in the corrector"}.get(int(mode[b]), "rule")
            row["jsplit"] = int(split[b])
        per_bucket.append(row)
    out = {"sweep": "powerlaw", "n": n, "t_end": DT_STEP, "wall_s": wall, "s_per_nbu": wall / DT_STEP,
           "block_steps": st["block_steps"], "particle_steps": st["particle_steps"],
           "interactions_per_s": (st["interactions"] - float(n) * n) / wall,
           "dE_E": abs((K1 + U1 - K0 - U0) / (K0 + U0)), "fused_path": fused, "histogram": per_bucket}
    print(json.dumps(out))
    return 0


def sweep_accuracy(a):
    """N = 16384 Plummer to t = 1 in the FP64 and mixed GPU forms: wall time per
    N-body unit and |dE/E| at t = 1."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    n = 16384
    m, x, v = inputs.plummer(n, seed=1)
    res = {}
    for prec in ("mixed", "fp64"):
        g = gravidy.Integrator(m, x, v, EPS, ETA, precision=prec)
        K0, U0 = g.energy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.evolve(1.0)
        wall = time.perf_counter() - t0
        K1, U1 = g.energy()
        st = g.stats()
        g.close()
        res[prec] = {"s_per_nbu": wall, "dE_E": abs((K1 + U1 - K0 - U0) / (K0 + U0)),
                     "block_steps": st["block_steps"], "particle_steps": st["particle_steps"]}
    # the N = 512 sphere of the first configuration to t = 1: both GPU forms and the oracle
    import oracle

    oracle.build()
    m, x, v = inputs.plummer(512, seed=1)
    small = {}
    for prec in ("mixed", "fp64"):
        g = gravidy.Integrator(m, x, v, EPS, ETA, precision=prec)
        E0 = sum(g.energy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.evolve(1.0)
        wall = time.perf_counter() - t0
        st = g.stats()
        small[prec] = {"s_per_nbu": wall, "dE_E": abs((sum(g.energy()) - E0) / E0),
                       "block_steps": st["block_steps"], "particle_steps": st["particle_steps"]}
        g.close()
    sim = oracle.Sim(m, x, v, EPS, ETA)
    E0 = sum(sim.energy())
    t0 = time.perf_counter()
    sim.evolve(1.0)
    so = sim.stats()
    small["oracle"] = {"s_per_nbu": time.perf_counter() - t0, "dE_E": abs((sum(sim.energy()) - E0) / E0),
                       "block_steps": so["nblock"], "particle_steps": so["nsteps"], "cores": 1}
    print(json.dumps({"sweep": "accuracy", "n": n, "t_end": 1.0, **res, "n512": small}))
    return 0


def sweep_ensemble(a):
    """256 independent Plummer spheres, N_c log-uniform in [256, 8192] (seeded),
    eps = 1e-4, eta = 0.01, mixed: advanced together as one ensemble (each system in
    its own thread-block cluster, the default; and the global-block-time forms: two
    kernels per global step, the cooperative kernel) vs the same clusters one after
    another (one context each, captured-graph steps)."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    sizes = inputs.ensemble_sizes(256, seed=1)
    ms, xs, vs = [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(int(n), seed=1000 + q)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    t_end = a.ens_t
    t_cmp = min(DT_STEP, t_end)  # every cluster compared with the oracle here
    e = gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA)
    K0, U0 = e.energy()
    s0 = e.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.evolve(t_cmp)
    wall_ens = time.perf_counter() - t0
    st_cmp = e.state()  # every particle at t_cmp (a multiple of dt_max)
    if t_end > t_cmp:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e.evolve(t_end)
        wall_ens += time.perf_counter() - t0
    K1, U1 = e.energy()
    s1 = e.stats()
    e.close()
    de = np.abs((K1 + U1 - K0 - U0) / (K0 + U0))
    wall_seq = 0.0
    inter_seq = 0.0
    steps_seq = 0
    for q in range(len(sizes)):
        g = gravidy.Integrator(ms[q], xs[q], vs[q], EPS, ETA, precision="mixed")
        st0 = g.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.evolve(t_end)
        wall_seq += time.perf_counter() - t0
        st1 = g.stats()
        inter_seq += st1["interactions"] - st0["interactions"]
        steps_seq += st1["block_steps"] - st0["block_steps"]
        g.close()
    inter_ens = s1["interactions"] - s0["interactions"]
    # the global-block-time form: two kernels per global step in a captured graph
    e = gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA, cluster=False)
    sg0 = e.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e.evolve(t_end)
    wall_g = time.perf_counter() - t0
    sg1 = e.stats()
    Kg, Ug = e.energy()
    e.close()
    two_kernel = {"wall_s": wall_g, "global_block_steps": sg1["block_steps"] - sg0["block_steps"],
                  "particle_steps": sg1["particle_steps"] - sg0["particle_steps"],
                  "interactions_per_s": (sg1["interactions"] - sg0["interactions"]) / wall_g,
                  "max_rel_energy_difference_vs_systems": float(np.max(np.abs((Kg + Ug) - (K1 + U1)) / np.abs(K1 + U1)))}
    # the cooperative form: select and force + correction of a global step in one
    # launch with a grid barrier between them, one step or 64 steps per launch
    fused = {}
    for spl in (1, 64):
        e = gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA,
                             fused=True, graph_steps=spl)
        sf0 = e.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e.evolve(t_end)
        wf = time.perf_counter() - t0
        sf1 = e.stats()
        e.close()
        fused["steps_per_launch_%d" % spl] = {
            "wall_s": wf, "global_block_steps": sf1["block_steps"] - sf0["block_steps"],
            "interactions_per_s": (sf1["interactions"] - sf0["interactions"]) / wf,
            "same_steps_as_two_kernel": sf1["block_steps"] - sf0["block_steps"] == two_kernel["global_block_steps"]}
    out = {"sweep": "ensemble", "clusters": int(sizes.size), "particles": int(sizes.sum()),
           "n_min": int(sizes.min()), "n_max": int(sizes.max()), "t_end": t_end,
           "ensemble": {"wall_s": wall_ens, "path": "independent systems (one thread-block cluster each)",
                        "system_block_steps": s1["block_steps"] - s0["block_steps"],
                        "particle_steps": s1["particle_steps"] - s0["particle_steps"],
                        "interactions_per_s": inter_ens / wall_ens},
           "two_kernel_global_steps": two_kernel,
           "fused": fused,
           "one_by_one": {"wall_s": wall_seq, "block_steps": steps_seq, "interactions_per_s": inter_seq / wall_seq},
           "speedup": wall_seq / wall_ens,
           "dE_E": {"median": float(np.median(de)), "max": float(de.max())}}
    # every cluster through the oracle to t_cmp on all host cores (one cluster per
    # worker at a time), with the energy error of the oracle's run and of the GPU
    # ensemble's state at t_cmp, both from the oracle's FP64 energy function
    cores = _host_cores()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    cjobs = [(q, int(nq), 1000 + q, t_cmp, st_cmp["x"][offs[q]:offs[q + 1]], st_cmp["v"][offs[q]:offs[q + 1]])
             for q, nq in enumerate(sizes)]
    cjobs.sort(key=lambda j: -j[1])  # large clusters first
    t0 = time.perf_counter()
    with _pool(cores) as pool:
        cres = pool.map(_oracle_compare_job, cjobs, chunksize=1)
    wall_cmp = time.perf_counter() - t0
    cres.sort(key=lambda r: r[0])
    de_gpu = np.array([r[3] for r in cres])
    de_or = np.array([r[4] for r in cres])
    ratio = de_gpu / np.maximum(de_or, 1e-300)
    within2 = de_gpu <= 2 * de_or + 1e-12
    big = de_or >= 1e-9  # above the floor the FP32 force arithmetic sets on a short run
    worst = int(np.argmax(ratio))
    out["per_cluster_vs_oracle"] = {
        "t": t_cmp, "clusters": len(cres), "energy": "oracle FP64 energy function on both states",
        "dE_E_gpu": {"median": float(np.median(de_gpu)), "max": float(de_gpu.max())},
        "dE_E_oracle": {"median": float(np.median(de_or)), "max": float(de_or.max())},
        "ratio_gpu_over_oracle": {"median": float(np.median(ratio)), "p5": float(np.percentile(ratio, 5)),
                                  "p95": float(np.percentile(ratio, 95)), "max": float(ratio.max())},
        "within_2x": int(within2.sum()),
        "oracle_dE_at_least_1e-9": {"clusters": int(big.sum()), "within_2x": int((within2 & big).sum()),
                                    "ratio_max": float(ratio[big].max()) if big.any() else None},
        "outside_2x": [{"cluster": int(q), "n": int(sizes[q]), "dE_E_gpu": float(de_gpu[q]),
                        "dE_E_oracle": float(de_or[q])} for q in np.nonzero(~within2)[0]],
        "worst": {"cluster": worst, "n": int(sizes[worst]), "dE_E_gpu": float(de_gpu[worst]),
                  "dE_E_oracle": float(de_or[worst])}}
    # the oracle's rate: all host cores over the comparison runs, and every 8th
    # cluster on one core to t = 1/64
    inter_all = sum(r[1] for r in cres)
    t_cpu = 1.0 / 64
    jobs = [(q, int(nq), 1000 + q, t_cpu) for q, nq in enumerate(sizes)]
    t0 = time.perf_counter()
    one = [_oracle_cluster_job(j) for j in jobs[::8]]
    wall_one = time.perf_counter() - t0
    out["oracle"] = {"all_cores": {"cores": cores, "clusters": len(cres), "t_end": t_cmp, "wall_s": wall_cmp,
                                   "interactions_per_s": inter_all / wall_cmp,
                                   "sample": "each cluster from t = 0 (its initial O(N_c^2) force included) to "
                                             "t = 1/8, plus two FP64 energies per cluster"},
                     "one_core": {"clusters": len(jobs[::8]), "t_end": t_cpu, "wall_s": wall_one,
                                  "interactions_per_s": sum(r[0] for r in one) / wall_one}}
    print(json.dumps(out))
    return 0


def sweep_eta(a):
    """Accuracy and cost against Aarseth's eta (the paper's eta sweep, Sec. 3.2):
    Plummer N = 1024, 4096, 16384 (seed 1, eps = 1e-4) integrated to t = 2 for
    eta = 0.001 .. 0.1 in mixed precision; at eta = 0.01 also the FP64 form and the
    distribution of block steps at t = 2 (the paper's step histogram); at N = 1024
    the oracle's |dE/E| for eta = 0.01 and 0.1."""
    import torch

    import oracle
    from paper_1702_00440_gb300 import gravidy, inputs

    t_end = 2.0
    rows = []
    for n in (1024, 4096, 16384):
        m, x, v = inputs.plummer(n, seed=1)
        for eta in (0.001, 0.003, 0.01, 0.03, 0.1):
            for prec in (("mixed", "fp64") if eta == 0.01 else ("mixed",)):
                g = gravidy.Integrator(m, x, v, EPS, eta, precision=prec, autotune=True)
                K0, U0 = g.energy()
                s0 = g.stats()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g.evolve(t_end)
                wall = time.perf_counter() - t0
                K1, U1 = g.energy()
                s1 = g.stats()
                row = {"n": n, "eta": eta, "precision": prec, "s_per_nbu": wall / t_end,
                       "dE_E": abs((K1 + U1 - K0 - U0) / (K0 + U0)),
                       "block_steps": s1["block_steps"] - s0["block_steps"],
                       "particle_steps": s1["particle_steps"] - s0["particle_steps"]}
                if eta == 0.01 and prec == "mixed":
                    lg = np.log2(g.state()["dtau"] * 2.0 ** -22).astype(int)
                    row["log2_dt_histogram"] = {int(b): int((lg == b).sum()) for b in np.unique(lg)}
                g.close()
                rows.append(row)
    oracle.build()
    m, x, v = inputs.plummer(1024, seed=1)
    orc = []
    for eta in (0.01, 0.1):
        sim = oracle.Sim(m, x, v, EPS, eta)
        E0 = sum(sim.energy())
        t0 = time.perf_counter()
        sim.evolve(t_end)
        orc.append({"n": 1024, "eta": eta, "dE_E": abs((sum(sim.energy()) - E0) / E0),
                    "wall_s": time.perf_counter() - t0, "block_steps": sim.stats()["nblock"]})
    print(json.dumps({"sweep": "eta", "t_end": t_end, "eps": EPS, "rows": rows, "oracle": orc}))
    return 0


def sweep_soft(a):
    """Accuracy and cost against the Plummer softening (the paper's softening sweep,
    Sec. 4.1): N = 1024, 4096, 16384 (seed 1) to t = 2 at eta = 0.01 for eps = 1e-5,
    1e-4, 1e-3, 1e-2, mixed precision; the oracle at N = 1024."""
    import torch

    import oracle
    from paper_1702_00440_gb300 import gravidy, inputs

    t_end = 2.0
    rows = []
    for n in (1024, 4096, 16384):
        m, x, v = inputs.plummer(n, seed=1)
        for eps in (1e-5, 1e-4, 1e-3, 1e-2):
            g = gravidy.Integrator(m, x, v, eps, ETA, precision="mixed", autotune=True)
            K0, U0 = g.energy()
            s0 = g.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.evolve(t_end)
            wall = time.perf_counter() - t0
            K1, U1 = g.energy()
            s1 = g.stats()
            g.close()
            rows.append({"n": n, "eps": eps, "s_per_nbu": wall / t_end, "dE_E": abs((K1 + U1 - K0 - U0) / (K0 + U0)),
                         "block_steps": s1["block_steps"] - s0["block_steps"],
                         "particle_steps": s1["particle_steps"] - s0["particle_steps"]})
    oracle.build()
    m, x, v = inputs.plummer(1024, seed=1)
    orc = []
    for eps in (1e-5, 1e-2):
        sim = oracle.Sim(m, x, v, eps, ETA)
        E0 = sum(sim.energy())
        t0 = time.perf_counter()
        sim.evolve(t_end)
        orc.append({"n": 1024, "eps": eps, "dE_E": abs((sum(sim.energy()) - E0) / E0),
                    "wall_s": time.perf_counter() - t0, "block_steps": sim.stats()["nblock"]})
    print(json.dumps({"sweep": "soft", "t_end": t_end, "eta": ETA, "rows": rows, "oracle": orc}))
    return 0


def sweep_lagrange(a):
    """Lagrange radii (radii enclosing 1, 5, 10, 25, 50, 75, 90 % of the mass about
    the centre of mass) of the N = 16384 benchmark sphere every 1/2 N-body unit to
    t = 8, with |dE/E| (the paper's Lagrange-radius diagnostic, Sec. 4.2, over a
    short stretch)."""
    from paper_1702_00440_gb300 import gravidy, inputs

    n = 16384
    m, x, v = inputs.plummer(n, seed=1)
    fr = np.array([0.01, 0.05, 0.1, 0.25, 0.5, 0.75, 0.9])

    def radii(xx):
        c = (m[:, None] * xx).sum(0) / m.sum()
        r = np.linalg.norm(xx - c, axis=1)
        o = np.argsort(r)
        cm = np.cumsum(m[o]) / m.sum()
        return [float(r[o][np.searchsorted(cm, f)]) for f in fr]

    g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", autotune=True)
    E0 = sum(g.energy())
    rows = [{"t": 0.0, "radii": radii(x), "dE_E": 0.0}]
    t0 = time.perf_counter()
    for k in range(1, 17):
        g.evolve(0.5 * k)
        rows.append({"t": 0.5 * k, "radii": radii(g.state()["x"]), "dE_E": abs((sum(g.energy()) - E0) / E0)})
    wall = time.perf_counter() - t0
    g.close()
    print(json.dumps({"sweep": "lagrange", "n": n, "fractions": fr.tolist(), "rows": rows, "wall_s": wall}))
    return 0


def density_centre(m, x, k=6):
    """Casertano & Hut (1985) density centre: positions weighted by the local
    density estimate m_i / r_k^3 (r_k the distance to the k-th nearest neighbour)."""
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    rk = np.sqrt(np.partition(d2, k, axis=1)[:, k])
    rho = m / rk ** 3
    return (rho[:, None] * x).sum(0) / rho.sum()


def lagrange_radii(m, x, fractions, centre):
    r = np.linalg.norm(x - centre, axis=1)
    o = np.argsort(r)
    cm = np.cumsum(m[o]) / m.sum()
    return [float(r[o][min(np.searchsorted(cm, f), len(r) - 1)]) for f in fractions]


def half_mass_relaxation_time(m, x):
    """t_rh = 0.138 (N r_h^3 / (G <m>))^(1/2) / ln(0.1 N), r_h the half-mass radius
    about the centre of mass (the paper's definition, Sec. 4.2; G = 1)."""
    n = len(m)
    c = (m[:, None] * x).sum(0) / m.sum()
    r_h = lagrange_radii(m, x, [0.5], c)[0]
    return 0.138 * math.sqrt(n * r_h ** 3 / m.mean()) / math.log(0.1 * n), r_h


COLLAPSE_FRACTIONS = [0.005, 0.01, 0.02, 0.05, 0.1, 0.25, 0.5, 0.75, 0.9]


def _collapse_rows(m, x, t_max, wall, evolve, energy, positions, block_steps):
    """The core-collapse diagnostics every 4 N-body units until t_max or `wall`
    seconds: Lagrange radii about the density centre, |dE/E|, block steps."""
    E0 = energy()
    rows = [{"t": 0.0, "radii": lagrange_radii(m, x, COLLAPSE_FRACTIONS, density_centre(m, x)), "dE_E": 0.0,
             "block_steps": 0, "wall_s": 0.0}]
    t0 = time.perf_counter()
    k = 0
    while True:
        k += 1
        t = 4.0 * k
        if t > t_max or time.perf_counter() - t0 > wall:
            break
        evolve(t)
        xs = positions()
        rows.append({"t": t, "radii": lagrange_radii(m, xs, COLLAPSE_FRACTIONS, density_centre(m, xs)),
                     "dE_E": abs((energy() - E0) / E0), "block_steps": block_steps(),
                     "wall_s": time.perf_counter() - t0})
    return rows


def _oracle_collapse_job(job):
    """One seed of the collapse sweep through the FP64 oracle on a host core."""
    seed, trh_factor, wall = job
    import oracle
    from paper_1702_00440_gb300 import inputs

    n = 1024
    m, x, v = inputs.plummer(n, seed=seed)
    trh, rh = half_mass_relaxation_time(m, x)
    sim = oracle.Sim(m, x, v, EPS, ETA)
    rows = _collapse_rows(m, x, trh_factor * trh, wall, sim.evolve, lambda: sum(sim.energy()),
                          lambda: sim.state()["x"], lambda: sim.stats()["nblock"])
    return {"sweep": "collapse", "impl": "oracle", "n": n, "seed": seed, "eps": EPS, "eta": ETA, "t_rh": trh,
            "r_h": rh, "fractions": COLLAPSE_FRACTIONS, "rows": rows}


def sweep_collapse(a):
    """Core collapse of an equal-mass Plummer sphere (N = 1024, eps = 1e-4, eta =
    0.01, mixed path; the paper's single-mass experiment, Sec. 4.2, at a size one
    GPU finishes in minutes): Lagrange radii about the density centre, |dE/E|,
    block steps and wall time every 4 N-body units, until t = --collapse-trh
    half-mass relaxation times or --collapse-wall seconds of wall time, for each
    seed of --collapse-seeds (one JSON line per seed).  --collapse-oracle runs
    the same diagnostics on the FP64 oracle instead, one seed per host core."""
    seeds = [int(q) for q in a.collapse_seeds.split(",")]
    if a.collapse_oracle:
        jobs = [(s, a.collapse_trh, a.collapse_wall) for s in seeds]
        with _pool(min(len(jobs), _host_cores())) as p:
            for res in p.imap(_oracle_collapse_job, jobs):
                print(json.dumps(res), flush=True)
        return 0
    from paper_1702_00440_gb300 import gravidy, inputs

    n = 1024
    for seed in seeds:
        m, x, v = inputs.plummer(n, seed=seed)
        trh, rh = half_mass_relaxation_time(m, x)
        g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", autotune=True)
        rows = _collapse_rows(m, x, a.collapse_trh * trh, a.collapse_wall, g.evolve, lambda: sum(g.energy()),
                              lambda: g.state()["x"], lambda: g.stats()["block_steps"])
        g.close()
        print(json.dumps({"sweep": "collapse", "impl": "gpu mixed", "n": n, "seed": seed, "eps": EPS, "eta": ETA,
                          "t_rh": trh, "r_h": rh, "fractions": COLLAPSE_FRACTIONS, "rows": rows}), flush=True)
    return 0


CLUSTER_PHASES = ("predict and list own active particles", "count push, barrier B1, offsets",
                  "gather the active records (DSMEM)", "force tasks", "segment sums and partial push",
                  "barrier B2", "correction (owners)", "minimum push, barrier B3", "next block time")


def sweep_cluster(a):
    """The small-step cluster's phase counters over one N-body unit of the
    benchmark workload (t = 0.375 -> 1.375, autotuned table), per small step, with
    the SM clock sampled meanwhile; and the CUDA-event time per cluster launch."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    gravidy.load()
    n = a.n
    m, x, v = inputs.plummer(n, seed=1)
    g = gravidy.Integrator(m, x, v, EPS, ETA, precision="mixed", autotune=True, time_force=True)
    g.evolve(0.375)
    g.kernel_time()
    g.cluster_time()
    c0, khz = g.cluster_phases()
    s0 = g.stats()
    sampler = ClockSampler(0)
    sampler.start()
    g.evolve(1.375)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    c1, _ = g.cluster_phases()
    s1 = g.stats()
    cms, cl = g.cluster_time()
    fms, fl, fi = g.kernel_time()
    info = g.cluster_info()
    g.close()
    d = c1 - c0
    steps = d[11]
    mhz = clocks["sm_mhz"] if clocks else khz / 1e3
    us = lambda cyc: cyc / (mhz * 1e6) * 1e6
    per = {name: us(d[k]) / max(steps, 1) for k, name in enumerate(CLUSTER_PHASES)}
    out = {"sweep": "cluster", "n": n, "t": [0.375, 1.375], "cluster_info": info, "small_steps": int(steps),
           "block_steps": s1["block_steps"] - s0["block_steps"], "sm_mhz": mhz, "clocks": clocks,
           "per_small_step_us": per, "per_small_step_total_us": sum(per.values()),
           "per_launch_us": {"prologue": us(d[9]) / max(cl, 1), "epilogue": us(d[10]) / max(cl, 1),
                             "cuda_events": 1e3 * cms / max(cl, 1)},
           "cluster_launches": cl, "force_launches": fl, "force_ms_per_launch": fms / max(fl, 1)}
    print(json.dumps(out))
    return 0


def sweep_fp32peak(a):
    """FP32 FMA throughput measured by the library's probe kernel (8 independent
    FMA chains per thread, every SM at full occupancy), repeated for about two
    seconds with the SM clock sampled meanwhile; the unit-count formula
    152 SMs x 128 lanes x 2 flop x f_SM is printed beside it at the sampled clock
    and at the maximum clock."""
    import torch

    from paper_1702_00440_gb300 import gravidy

    gravidy.load()
    torch.cuda.set_device(0)
    gravidy.gd_probe_fma(0, 1 << 12)
    sampler = ClockSampler(0)
    sampler.start()
    runs = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 2.0:
        runs.append(gravidy.gd_probe_fma(0, 1 << 18))
    clocks = sampler.stop()
    best = max(r[0] for r in runs)
    med = statistics.median(r[0] for r in runs)
    mhz = clocks["sm_mhz"] if clocks else None
    out = {"sweep": "fp32peak", "probe_tflops_best": best, "probe_tflops_median": med, "probes": len(runs),
           "ms_per_probe": statistics.median(r[1] for r in runs), "clocks": clocks,
           "formula_tflops_at_max_clock": FP32_PEAK_TFLOPS,
           "formula_tflops_at_sampled_clock": (SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12) if mhz else None,
           "probe_over_formula_at_sampled_clock": (best / (SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12)) if mhz else None}
    print(json.dumps(out))
    return 0


def sweep_h6(a):
    """Sixth- against fourth-order Hermite on Plummer N = 1024 and 4096 (seed 1,
    eps = 1e-4) to t = 1: wall time per N-body unit and |dE/E| for the FP64
    fourth-order path at eta = 0.003, 0.01, 0.03, the FP64 sixth-order path at
    eta = 0.1, 0.2, 0.4 and the mixed fourth-order path at eta = 0.003, 0.01;
    and full force/jerk/snap evaluations (N = 16384, 65536) of the sixth-order
    kernel."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    rows = []
    for n in (1024, 4096):
        m, x, v = inputs.plummer(n, seed=1)
        runs = [("h4", "fp64", e) for e in (0.003, 0.01, 0.03)] + [("h6", "fp64", e) for e in (0.1, 0.2, 0.4)] + \
               [("h4", "mixed", e) for e in (0.003, 0.01)]
        for order, prec, eta in runs:
            if order == "h6":
                g = gravidy.Integrator6(m, x, v, EPS, eta)
            else:
                g = gravidy.Integrator(m, x, v, EPS, eta, precision=prec, autotune=prec == "mixed")
            E0 = sum(g.energy())
            s0 = g.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.evolve(1.0)
            wall = time.perf_counter() - t0
            E1 = sum(g.energy())
            s1 = g.stats()
            g.close()
            rows.append({"n": n, "order": order, "precision": prec, "eta": eta, "s_per_nbu": wall,
                         "dE_E": abs((E1 - E0) / E0), "block_steps": s1["block_steps"] - s0["block_steps"],
                         "particle_steps": s1["particle_steps"] - s0["particle_steps"]})
    force = []
    for n in (16384, 65536):
        m, x, v = inputs.plummer(n, seed=1)
        with gravidy.Integrator6(m, x, v, EPS, 0.2) as g:
            idx = np.arange(n, dtype=np.int32)
            g.force(0, idx)
            t0 = time.perf_counter()
            g.force(0, idx)
            dt = time.perf_counter() - t0
        force.append({"n": n, "s": dt, "interactions_per_s": float(n) * n / dt})
    print(json.dumps({"sweep": "h6", "t_end": 1.0, "eps": EPS, "rows": rows, "force": force}))
    return 0


def sweep_timesym(a):
    """The time-symmetric schemes of the gd_h6 engine.  (1) Plummer N = 1024 and
    4096 (seed 1, eps = 1e-4) to t = 1: wall time per N-body unit, |dE/E| and
    step counts of GraviDy's FP64 fourth-order path (eta = 0.01), the
    time-symmetric fourth-order corrector with one and two passes (eta = 0.01)
    and the sixth-order scheme with one and two passes (eta = 0.2).  (2) The
    e = 0.5 Kepler orbit with shared constant steps (dt_min = dt_max): the mean
    energy error of each of 8 orbits, its linear drift over the run relative to
    its mean, and the distance from the start after one orbit forward and back
    with reversed velocities."""
    import torch

    from paper_1702_00440_gb300 import gravidy, inputs

    rows = []
    for n in (1024, 4096):
        m, x, v = inputs.plummer(n, seed=1)
        runs = [("h4 standard", 4, 0, 0.01), ("h4 time-symmetric", 4, 1, 0.01), ("h4 time-symmetric", 4, 2, 0.01),
                ("h6", 6, 1, 0.2), ("h6", 6, 2, 0.2)]
        for name, order, n_iter, eta in runs:
            if n_iter == 0:
                g = gravidy.Integrator(m, x, v, EPS, eta, precision="fp64")
            else:
                g = gravidy.Integrator6(m, x, v, EPS, eta, eta_init=eta if order == 4 else 0.001, order=order,
                                        n_iter=n_iter)
            E0 = sum(g.energy())
            s0 = g.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.evolve(1.0)
            wall = time.perf_counter() - t0
            E1 = sum(g.energy())
            s1 = g.stats()
            g.close()
            rows.append({"n": n, "scheme": name, "n_iter": max(n_iter, 1), "eta": eta, "s_per_nbu": wall,
                         "dE_E": abs((E1 - E0) / E0), "block_steps": s1["block_steps"] - s0["block_steps"],
                         "particle_steps": s1["particle_steps"] - s0["particle_steps"],
                         "interactions": s1["interactions"] - s0["interactions"]})
    # Kepler binary, G = M = 1, semi-major axis 1, e = 0.5, at pericentre at t = 0
    e = 0.5
    rp = 1.0 - e
    vp = math.sqrt((1 + e) / rp)
    mk = np.array([0.5, 0.5])
    xk = np.array([[-rp / 2, 0, 0], [rp / 2, 0, 0]])
    vk = np.array([[0, -vp / 2, 0], [0, vp / 2, 0]])
    kepler = []
    for order, dt in ((4, 2.0 ** -8), (6, 2.0 ** -7)):
        nper = int(round(2 * math.pi / dt))
        for n_iter in (1, 2):
            with gravidy.Integrator6(mk, xk, vk, 0.0, 0.2, order=order, n_iter=n_iter, dt_min=dt, dt_max=dt) as g:
                E0 = sum(g.energy())
                err = []
                for _ in range(8 * nper):
                    g.step_block()
                    err.append(sum(g.energy()) / E0 - 1)
            means = np.array(err).reshape(8, nper).mean(axis=1)
            drift = abs(np.polyfit(np.arange(8), means, 1)[0]) * 7 / abs(means.mean())
            t1 = nper * dt
            with gravidy.Integrator6(mk, xk, vk, 0.0, 0.2, order=order, n_iter=n_iter, dt_min=dt, dt_max=dt) as g:
                g.evolve(t1)
                fw = g.state()
            with gravidy.Integrator6(mk, fw["x"], -fw["v"], 0.0, 0.2, order=order, n_iter=n_iter, dt_min=dt,
                                     dt_max=dt) as g:
                g.evolve(t1)
                bk = g.state()
            back = max(np.abs(bk["x"] - xk).max(), np.abs(bk["v"] + vk).max())
            kepler.append({"order": order, "n_iter": n_iter, "dt": dt, "orbit_mean_dE_E": [float(q) for q in means],
                           "drift_over_8_orbits_rel_to_mean": float(drift), "round_trip_one_orbit": float(back)})
    print(json.dumps({"sweep": "timesym", "t_end": 1.0, "eps": EPS, "rows": rows, "kepler": kepler}))
    return 0


def profile_force(a):
    from paper_1702_00440_gb300 import gravidy, inputs

    m, x, v = inputs.plummer(a.profile_force, seed=1)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=a.precision) as g:
        g.force(0, np.arange(a.profile_force, dtype=np.int32))
    return 0


def profile_force_h6(a):
    from paper_1702_00440_gb300 import gravidy, inputs

    m, x, v = inputs.plummer(a.profile_force_h6, seed=1)
    with gravidy.Integrator6(m, x, v, EPS, 0.2) as g:
        g.force(0, np.arange(a.profile_force_h6, dtype=np.int32))
    return 0


def profile_steps(a):
    """Integrates to t = 0.375 (the start of the timed window), then runs the next
    1/64 N-body time unit between cudaProfilerStart/Stop, so that
    `ncu --profile-from-start off` sees only steady-state block steps."""
    import torch
    from paper_1702_00440_gb300 import gravidy, inputs

    m, x, v = inputs.plummer(a.n, seed=1)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=a.precision, autotune=True) as g:
        g.evolve(0.375)
        s0 = g.stats()
        torch.cuda.profiler.start()
        g.evolve(0.375 + a.profile_steps / 64.0)
        torch.cuda.profiler.stop()
        s1 = g.stats()
        print(json.dumps({"block_steps": s1["block_steps"] - s0["block_steps"],
                          "kernel_launches": s1["kernel_launches"] - s0["kernel_launches"]}))
    return 0


def profile_ensemble(a):
    """The first K clusters of the ensemble workload (seeded sizes, Plummer), advanced
    to t = 1/64 with the default (independent-cluster) path between
    cudaProfilerStart/Stop; prints the wall time and the counters."""
    import torch
    from paper_1702_00440_gb300 import gravidy, inputs

    sizes = inputs.ensemble_sizes(256, seed=1)[:a.profile_ensemble]
    ms, xs, vs = [], [], []
    for q, n in enumerate(sizes):
        m, x, v = inputs.plummer(int(n), seed=1000 + q)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    with gravidy.Ensemble(sizes, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs), EPS, ETA) as e:
        s0 = e.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        torch.cuda.profiler.start()
        e.evolve(1.0 / 64)
        torch.cuda.profiler.stop()
        wall = time.perf_counter() - t0
        s1 = e.stats()
    print(json.dumps({"clusters": int(sizes.size), "particles": int(sizes.sum()), "wall_s": wall,
                      "interactions_per_s": (s1["interactions"] - s0["interactions"]) / wall,
                      "block_steps": s1["block_steps"] - s0["block_steps"]}))
    return 0


def profile_nact(a):
    import torch
    from paper_1702_00440_gb300 import gravidy, inputs

    m, x, v = inputs.plummer(a.n, seed=1)
    with gravidy.Integrator(m, x, v, EPS, ETA, precision=a.precision, autotune=True) as g:
        mc, split, mode, ms = g.tuning()
        nb = int(np.log2(a.n)) + 1
        print(json.dumps({"n": a.n, "split": split[:nb].tolist(), "mode": mode[:nb].tolist(),
                          "us": [round(1e3 * float(t), 2) for t in ms[:nb]]}))
        idx = inputs.random_subset(a.n, a.profile_nact, seed=5)
        g.force(0, idx)
        torch.cuda.profiler.start()
        g.force(0, idx)
        g.force(0, idx)
        torch.cuda.profiler.stop()
    return 0


def main():
    a = _args()
    if a.profile_nact:
        return profile_nact(a)
    if a.profile_force:
        return profile_force(a)
    if a.profile_force_h6:
        return profile_force_h6(a)
    if a.profile_steps:
        return profile_steps(a)
    if a.profile_ensemble:
        return profile_ensemble(a)
    if a.sweep:
        return {"force": sweep_force, "powerlaw": sweep_powerlaw, "accuracy": sweep_accuracy,
                "ensemble": sweep_ensemble, "eta": sweep_eta, "soft": sweep_soft,
                "lagrange": sweep_lagrange, "h6": sweep_h6,
            "timesym": sweep_timesym, "collapse": sweep_collapse, "fp32peak": sweep_fp32peak,
            "cluster": sweep_cluster}[a.sweep](a)
    if a.impl == "reference":
        return run_reference(a)
    return run_gravidy(a)


if __name__ == "__main__":
    sys.exit(main())
