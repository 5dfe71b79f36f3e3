"""One rank of the replica-aggregation check (launched by tests/test_replicas.py
through torch.distributed.run, gloo backend, on the CPU): every rank reports a
different time; each must see the slowest one and the same whole-job rate."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = bench.max_over_ranks(10.0 + 3.0 * rank, dist)
rate = bench.job_rate(1000.0, world, t)
dist.barrier()
with open(os.path.join(os.environ["REPLICA_OUT"], f"rank{rank}.json"), "w") as f:
    json.dump({"rank": rank, "world": world, "t": t, "rate": rate}, f)
dist.destroy_process_group()
