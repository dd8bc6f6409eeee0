"""The multi-rank path of bench.py on CPU: two gloo ranks.

Under torchrun every rank runs its own ParRep instances on its own GPU with
no collective on the data path; only the figures are combined: the job's
time is the slowest rank's, the event counts add up, and no two ranks share
a seed.  This checks that host logic with the gloo backend (no GPU).
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_rank = 1.5 + rank                       # seconds this rank timed
    counts = [1000 * (rank + 1), 7 + rank]   # useful, executed
    t, c = bench.combine_ranks(dist, t_rank, counts, "cpu")
    seeds = [bench.rank_seed(rank, i) for i in range(8)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (t, c, gathered)
    dist.destroy_process_group()


def test_two_ranks_combine_time_and_counts():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, c, gathered = res[rank]
        assert t == pytest.approx(2.5)          # the slowest rank
        assert c == [3000, 15]                  # sums over ranks
        all_seeds = [s for g in gathered for s in g]
        assert len(set(all_seeds)) == len(all_seeds)


def test_single_process_combine_is_identity():
    import bench

    assert bench.combine_ranks(None, 3.25, [10, 20], "cpu") == (3.25, [10, 20])
