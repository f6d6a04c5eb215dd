"""One rank of a replica job on the host (run by tests/test_replicas_gloo.py
through replicas.spawn, the launcher bench.py uses for --gpus N): every
rank analyses its own seeded frame pair with the oracle, the ranks take the
max of their times over gloo, and rank 0 prints the whole-job line."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_12191_gb300 import replicas, synth  # noqa: E402


def main():
    rank, world, local = replicas.env()
    replicas.init("gloo")
    seed = replicas.seed_base(rank)
    fp = synth.frame_pair(seed, 128, 64, 8)
    replicas.barrier()
    t0 = time.perf_counter()
    out = oracle.analyze(fp.cur, fp.ref, qp=30, search_range=8, threads=1)
    dt = replicas.max_over_ranks(time.perf_counter() - t0)
    evaluated = replicas.sum_over_ranks(int(sum(int(e.sum()) for e in out["evaluated"])))
    if rank == 0:
        print(json.dumps({"n_gpus": world, "value": replicas.job_rate(1, world, dt), "unit": "frames/s",
                          "evaluated_cus": evaluated, "seed_rank0": seed}))
    replicas.barrier()
    replicas.finish()


if __name__ == "__main__":
    main()
