"""Host-side multi-rank path of bench.py with world_size 2 on CPU (gloo): each
rank owns a distinct catalog shard, and timings are reduced with a max so the
reported rate is whole-job events over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import gwcat
    raw = gwcat.draw("c3", 50, seed=bench.shard_seed(rank))
    my_times = [10.0 * (rank + 1), 20.0 * (rank + 1), 1.0 + rank]
    t, rates = bench.aggregate(my_times, 50, 4, world, dist)
    digest = torch.tensor(raw["m1"][:5], dtype=torch.float64)
    gathered = [torch.zeros(5, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (t, rates, [g.numpy().tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    t0, rates0, g0 = res[0]
    t1, rates1, g1 = res[1]
    assert t0 == t1 == [20.0, 40.0, 2.0]                       # max over ranks
    assert abs(rates0[0] - 2 * 50 * 4 / 0.020) < 1e-6          # whole-job events / max time
    assert not np.allclose(g0[0], g0[1])                       # distinct shards
