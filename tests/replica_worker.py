"""One rank of the replica-path test: runs bench.py's rendezvous and whole-job
aggregation under torch.distributed (gloo) and prints what it saw."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def main():
    args = bench.parse()
    rank, world, local = bench.dist_init(args)
    # every rank did the same 1e9 units; rank r took 1 + r seconds
    rate = bench.whole_job_rate(1e9, 1.0 + rank, world)
    mx = bench.max_over_ranks(float(rank) + 0.5, world)
    bench.barrier(world)
    print(json.dumps({"rank": rank, "world": world, "local": local, "rate": rate, "max": mx}))


if __name__ == "__main__":
    main()
