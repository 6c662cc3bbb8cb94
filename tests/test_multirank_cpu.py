"""The multi-rank bench path on CPU: two gloo ranks, disjoint instance
shards, max-over-ranks timing and the whole-job rate."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = wl.single_cell_64(8, base_seed=bench.rank_base_seed(rank), p_db=(10,))
    first = insts[0].H[0, 0, :4].copy()
    elapsed = 1.0 + rank          # rank 1 is the slowest
    slowest = bench.max_over_ranks(elapsed, dist)
    rate = bench.whole_job_rate(world, len(insts), 3, slowest)
    out[rank] = (slowest, rate, first)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0
    assert res[0][1] == pytest.approx(2 * 8 * 3 / 2.0)
    assert not np.allclose(res[0][2], res[1][2])   # disjoint shards
