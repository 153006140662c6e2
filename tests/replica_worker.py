"""One rank of the replicas-only multi-process check (launched by test_replicas_cpu.py
under torch.distributed.run with the gloo backend on CPU)."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo", init_method="env://")
    rank, world, _ = bench.dist_env()
    # Each replica times its own steps; the job's time is the slowest replica's.
    seconds = bench.max_over_ranks(1.5 * (rank + 1), world, device="cpu")
    rate = bench.whole_job_rate(100.0, 4, seconds, world)
    dist.barrier()
    if rank == 0:
        print(json.dumps({"world": world, "seconds": seconds, "rate": rate}), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
