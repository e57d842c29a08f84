"""The multi-GPU path's host logic on CPU, as two gloo ranks: evaluations are
sharded over replicas with no exchange on the data path (every direction on
exactly one rank), and the whole job is timed by the slowest rank (a max over
ranks), its value being all ranks' evaluations over that time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2608_07307_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        table = I.sun_dirs_fibonacci(4096)
        mine = bench.shard(table, rank, world)
        # every direction on exactly one rank
        sizes = torch.tensor([len(mine)], dtype=torch.int64)
        dist.all_reduce(sizes)
        ids = torch.zeros(len(table), dtype=torch.int64)
        for row in mine:
            ids[int(np.argmin(np.abs(table - row).sum(axis=1)))] += 1
        dist.all_reduce(ids)

        def reduce_max(xs):
            t = torch.tensor(xs, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return [float(x) for x in t]

        local_ms = 100.0 + 50.0 * rank
        local_e2e = 0.2 + 0.1 * rank
        total_ms, e2e_s, evals, value = bench.job_totals(local_ms, local_e2e, 320, world, reduce_max)
        dist.barrier()
        out[rank] = (int(sizes), int(ids.min()), int(ids.max()), total_ms, e2e_s, evals, value)
    finally:
        dist.destroy_process_group()


def test_replicas_shard_and_time_as_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        n, lo, hi, total_ms, e2e_s, evals, value = res[rank]
        assert n == 4096 and lo == 1 and hi == 1
        assert total_ms == 150.0 and e2e_s == pytest.approx(0.3)
        assert evals == 640 and value == pytest.approx(640 / 0.15)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    total_ms, e2e_s, evals, value = bench.job_totals(80.0, 0.1, 32, 1)
    assert (total_ms, e2e_s, evals) == (80.0, 0.1, 32) and value == pytest.approx(400.0)
    table = np.arange(12.0).reshape(4, 3)
    assert np.array_equal(bench.shard(table, 0, 1), table)
