"""Multi-GPU replicas on CPU: two gloo ranks run bench.py's job-level
reduction (slowest rank's time, summed counts) and its per-rank seeding, which
must give every replica its own Philox stream of RR sets."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 50.0 * rank  # the slower rank sets the job time
        counts = (1000 * (rank + 1), 10 * (rank + 1), 3 * (rank + 1))
        ms_max, totals = bench.reduce_over_ranks(ms, counts, "cpu")
        seeds = [bench.replica_seed(rank, s) for s in range(5)]
        everyone = [None] * world
        dist.all_gather_object(everyone, seeds)
        out[rank] = (ms_max, totals, everyone)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_seed():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, totals, everyone = res[rank]
        assert ms_max == 150.0
        assert totals == [3000.0, 30.0, 9.0]
        flat = [s for seeds in everyone for s in seeds]
        assert len(set(flat)) == len(flat)  # no two replicas or steps share a seed
