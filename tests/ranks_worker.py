"""Worker for the two-rank CPU test of bench.py's multi-rank host logic (launched by torchrun,
gloo backend, no GPU): each rank times its own independent batch, the job takes the slowest
rank's time and counts every rank's units."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    rank, world, _ = bench.dist_env()
    dist.init_process_group("gloo")
    ms = 10.0 + 5.0 * rank  # this rank's own step time
    slowest = bench.max_over_ranks(ms, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    rate = bench.job_rate(1000, 2, world, slowest)
    # one file per rank: the ranks' standard outputs share a pipe and can interleave
    with open(os.path.join(sys.argv[1], f"rank{rank}.json"), "w") as f:
        json.dump({"rank": rank, "world": world, "max_ms": slowest, "seeds": seeds, "rate": rate}, f)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
