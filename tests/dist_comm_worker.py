"""Worker for tests/test_bench_dist.py, launched by torch.distributed.run on the
CPU: bench.py's rank communicator over gloo (barrier, MAX and SUM reductions
and the whole-job rate the benchmark reports) with rank-dependent values."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main(out_dir):
    world, rank, _ = bench._dist()
    comm = bench._Comm(world, rank, False)
    comm.barrier()
    seconds = 1.0 + rank            # rank r takes 1 + r seconds
    units = 1000.0 * (rank + 1)     # and processes 1000 (r + 1) units
    res = {"rank": rank, "world": world, "backend": comm.dist.get_backend() if comm.dist else None,
           "max_s": comm.reduce(seconds, "MAX"), "sum_units": comm.reduce(units, "SUM")}
    res["rate"] = res["sum_units"] / res["max_s"]
    comm.barrier()
    comm.close()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)


if __name__ == "__main__":
    main(sys.argv[1])
