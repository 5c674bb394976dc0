"""The N > 1 bookkeeping of bench.py on CPU ranks (gloo, world size 2):
every rank gets the slowest rank's time, throughput counts all ranks' work,
and replicas draw different inputs."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + 2.0 * rank)  # rank 1 is the slow one
    res = {"max": t, "seeds": bench.replica_seeds(rank),
           "throughput": bench.job_throughput(100.0, world, t)}
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as fh:
        json.dump(res, fh)


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{i}.json")) for i in range(2)]
    assert r[0]["max"] == r[1]["max"] == 3.0
    assert r[0]["throughput"] == r[1]["throughput"] == 2 * 100.0 / 3.0
    assert r[0]["seeds"] != r[1]["seeds"]


def _instance_worker(rank, world, port, out):
    """Each rank evaluates its share of batch instances with a host stand-in
    (the oracle's forward of a small lattice shaped like the instance)."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    from paper_2310_00810_gb300 import replicas as R

    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = _instances()
    res = R.run_sharded(items, _stand_in, costs=[nx * ny for nx, ny, _, _ in items])
    mine = R.shard([nx * ny for nx, ny, _, _ in items], world)[rank]
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"i{rank}.json"), "w") as fh:
        json.dump({"results": res, "mine": mine}, fh)


def _instances():
    from paper_2310_00810_gb300 import workloads as W

    return [(nx // 16, ny // 16, por, sd) for nx, ny, por, sd in W.batch_sizes(7, seed=4000)]


def _stand_in(item):
    import numpy as np

    from oracle import oracle as O
    from paper_2310_00810_gb300 import workloads as W

    nx, ny, _, sd = item
    m, _ = O.geometry(9, max(nx, 8), max(ny, 4))
    rin = 1.0 + W.inlet_profile(m.shape[0], seed=2000 + sd)
    _, u = O.macroscopic(9, m, O.forward(9, m, rin, 1.0, 0.8, 20))
    return [float(np.sum(u[0])), float(np.sum(u[1] ** 2))]


def test_ranks_split_instances_and_gather_the_one_rank_result(tmp_path):
    port = _free_port()
    mp.spawn(_instance_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"i{i}.json")) for i in range(2)]
    from paper_2310_00810_gb300 import replicas as R

    want = R.run_sharded(_instances(), _stand_in)  # one rank, no process group
    assert r[0]["results"] == r[1]["results"] == want
    assert sorted(r[0]["mine"] + r[1]["mine"]) == list(range(len(want)))
    assert r[0]["mine"] and r[1]["mine"] and not set(r[0]["mine"]) & set(r[1]["mine"])


def test_shard_balances_costs():
    from paper_2310_00810_gb300 import replicas as R

    costs = [9, 1, 8, 2, 7, 3, 6, 4, 5]
    parts = R.shard(costs, 3)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert sorted(i for p in parts for i in p) == list(range(9))
    assert loads == [16, 15, 14]  # the longest-processing-time assignment, deterministic
    assert max(loads) <= 4 / 3 * sum(costs) / 3  # LPT's bound against the best split
    assert R.shard(costs, 1) == [list(range(9))]
