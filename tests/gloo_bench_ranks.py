"""Helper run under torchrun by tests/test_bench_host.py: the multi-rank host logic of
bench.py on CPU ranks (gloo).  Each rank reports a different time; every rank must see
the max, and the whole-job value must count every rank's right-hand sides."""

import json
import os
import sys

import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    world, rank, _ = bench.dist_env()
    dist.init_process_group("gloo")
    per_rank_ms = 10.0 + 3.0 * rank
    ms = bench.reduce_max(per_rank_ms, torch.device("cpu"))
    value = bench.aggregate_value(world, 5, 4, ms / 1e3)
    mine = {"rank": rank, "world": world, "ms": ms, "value": value}
    every = [None] * world
    dist.all_gather_object(every, mine)        # rank 0 prints all lines: no interleaved output
    if rank == 0:
        sys.stdout.write("".join(json.dumps(r) + "\n" for r in every))
        sys.stdout.flush()
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
