"""The multi-rank path of bench.py (weak scaling: agents sharded over ranks,
no collective on the data path, job time = max over ranks) with two gloo
ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, steps, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = bench.shard_ids(n, rank, world)
    local_ms = 100.0 + 25.0 * rank                 # rank 1 is the slow one
    value, job_ms = bench.job_throughput(n, steps, local_ms, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, ids.tolist())
    if rank == 0:
        out.put((value, job_ms, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    world, n, steps, port = 2, 5, 4, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    value, job_ms, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert job_ms == 125.0                                    # max over ranks
    assert abs(value - world * n * steps / 0.125) < 1e-9      # whole-job agent-solves/s
    all_ids = np.concatenate(gathered)
    assert sorted(all_ids.tolist()) == list(range(world * n))  # disjoint, covering


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, job_ms = bench.job_throughput(7, 3, 50.0, 1)
    assert job_ms == 50.0 and abs(value - 7 * 3 / 0.05) < 1e-9
    assert list(bench.shard_ids(3, 2, 4)) == [6, 7, 8]
