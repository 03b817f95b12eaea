"""bench.py's multi-rank host logic on the CPU (world size 2, gloo), launched
the way the benchmark is launched for N > 1 (torch.distributed.run, one process
per rank, rendezvous on 127.0.0.1): the rank communicator's barrier and
reductions, the whole-job rate (units of all ranks over the slowest rank's
time), and the reference arm, which only rank 0 runs and prints."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=env)


def test_rank_communicator_over_gloo(tmp_path):
    out = _torchrun([os.path.join(ROOT, "tests", "dist_comm_worker.py"), str(tmp_path)])
    assert out.returncode == 0, out.stderr[-2000:]
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == 2 and d["backend"] == "gloo"
        assert d["max_s"] == 2.0 and d["sum_units"] == 3000.0
        assert d["rate"] == 1500.0


def test_reference_arm_under_two_ranks_prints_once():
    # (no --n: torch.distributed.run reads it as an ambiguous prefix of its own options)
    out = _torchrun([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2",
                     "--warmup", "1"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == 1
