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
