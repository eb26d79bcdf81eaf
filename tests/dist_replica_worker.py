"""One rank of the benchmark's replica path on CPU (gloo), run under torchrun by
tests/test_dist_cpu.py: every rank reports its own per-step times, the job
takes the max over ranks (the slowest replica), rank 0 alone prints."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    mine = [10.0 + rank, 50.0 - 3.0 * rank, 7.5 * (rank + 1)]
    dist.barrier()
    got = bench.max_over_ranks(mine, dist, "cpu")
    if rank == 0:
        print(json.dumps({"world": world, "max": got, "solves_per_s": world * 1e3 / got[0]}))
    dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
