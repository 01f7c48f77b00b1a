"""Multi-process path of bench.py (replicas, no data-path collective): the
step time is the max over ranks and the value sums all ranks' work.  Two gloo
ranks on CPU."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.reduce_step_time(100.0 + 50.0 * rank, world, dist, "cpu")
    out[rank] = (ms, bench.aggregate_value(world, 128 ** 3, 64, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    world, port = 2, 29531
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 150.0
        assert abs(value - 2 * 128 ** 3 * 64 / 0.150) < 1e-6 * value
