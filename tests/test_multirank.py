"""Host-side multi-rank path of bench.py with world_size 2 on CPU (gloo): each
rank owns a distinct catalog shard, timings are reduced with a max so the
reported rate is whole-job events over the slowest rank's time, and the one
data-path exchange, the log-det gradient of the summed log det (a sum over
events), is the all-reduced sum of the ranks' shard gradients."""
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


def _worker_logdet(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import gwcat
    import oracle
    from tests.helpers import oracle_catalog
    cat, _, _ = oracle_catalog("c4", world, max_npts=60)
    det, psd, rot = gwcat.network("c4")
    g, _ = oracle.logdet_grad_gamma(cat.subset(np.array([rank])), det, psd, rot, 11, [1, 2])
    t = torch.tensor(np.asarray(g), dtype=torch.float64)
    bench.sum_over_ranks(t, world, dist)
    out[rank] = t.tolist()
    dist.destroy_process_group()


def test_logdet_gradient_is_the_sum_over_shards():
    """The c4 log-det VJP on a catalog split over two ranks (one event each):
    the all-reduced shard gradients equal the whole catalog's gradient (the
    oracle's fixed-step Richardson differences are linear in the summed
    log det, so the sum is exact up to rounding)."""
    import gwcat
    import oracle
    from tests.helpers import oracle_catalog
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker_logdet, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    cat, _, _ = oracle_catalog("c4", world, max_npts=60)
    det, psd, rot = gwcat.network("c4")
    g_all, _ = oracle.logdet_grad_gamma(cat, det, psd, rot, 11, [1, 2])
    for r in range(world):
        np.testing.assert_allclose(res[r], g_all, rtol=1e-12, atol=0)
