"""Host-side multi-rank path with world_size 2 on CPU (gloo).

One catalog is split into contiguous ranges balanced by cost (grid points x
effective interferometers; the paper's index-range split of Sec. 5 over its
process pool or MPI ranks), every rank computes its range, and the results are
gathered back in catalog order; timings are reduced with a max, so the reported
rate is whole-job events over the slowest rank's time; the one data-path
exchange, the log-det gradient of the summed log det (a sum over events), is
the all-reduced sum of the ranks' shard gradients."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2207_06910_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("world", [1, 2, 3, 8, 64])
def test_partition_is_contiguous_and_balanced_to_one_event(world):
    rng = np.random.default_rng(world)
    for n in (1, 7, 1000, 100_000):
        npts = np.round(np.exp(rng.uniform(np.log(200), np.log(20000), n)))
        d_eff = rng.choice([2, 4], n)
        cost = shard.event_cost(npts, d_eff)
        b = shard.partition(cost, world)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
        assert shard.imbalance(cost, b) <= cost.max() * (1 + 1e-12)


def test_partition_uneven_catalog():
    """A catalog whose costs vary 100x (the stress grid) and a single dominant
    event: the ranges stay within one event's cost of the mean."""
    cost = np.concatenate([np.full(500, 200.0), [2e5], np.full(500, 2e4)])
    for world in (2, 4, 16):
        b = shard.partition(cost, world)
        assert shard.imbalance(cost, b) <= cost.max()
    with pytest.raises(ValueError):
        shard.partition(np.array([1.0, -1.0]), 2)


# ---------------------------------------------------------------- gather
def _worker_gather(rank, world, port, out):
    _init(rank, world, port)
    import gwcat
    import oracle
    from tests.helpers import oracle_catalog
    cat, _, _ = oracle_catalog("c1", 7, max_npts=40)
    det, psd, rot = gwcat.network("c1")
    b = shard.partition(shard.event_cost(cat.npts, 2), world)
    sub = cat.subset(np.arange(b[rank], b[rank + 1]))
    F, s, err, st = oracle.fisher(sub, det, psd, rot, 11)
    iu = np.triu_indices(11)
    local = {"fisher": F[:, iu[0], iu[1]].T.copy(), "snr": s, "status": st}
    got = shard.gather_events(local, b, rank, world, dist)
    out[rank] = None if got is None else {k: v.tolist() for k, v in got.items()}
    # timings: max over ranks; whole-job rate over the slowest rank
    import bench
    t, rates = bench.aggregate([10.0 * (rank + 1), 1.0 + rank], 7 * world, 4, world, dist)
    out[f"t{rank}"] = (t, rates)
    dist.destroy_process_group()


def test_two_ranks_gather_equals_one_process():
    """Two gloo ranks each run the oracle on their range of one catalog; the
    gathered results equal the one-process results bit for bit."""
    import gwcat
    import oracle
    from tests.helpers import oracle_catalog
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker_gather, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[1] is None
    cat, _, _ = oracle_catalog("c1", 7, max_npts=40)
    det, psd, rot = gwcat.network("c1")
    F, s, err, st = oracle.fisher(cat, det, psd, rot, 11)
    iu = np.triu_indices(11)
    assert np.array_equal(np.array(res[0]["fisher"]), F[:, iu[0], iu[1]].T)
    assert np.array_equal(np.array(res[0]["snr"]), s)
    assert np.array_equal(np.array(res[0]["status"]), st)
    t0, rates0 = res["t0"]
    t1, rates1 = res["t1"]
    assert t0 == t1 == [20.0, 2.0]                            # max over ranks
    assert abs(rates0[0] - 2 * 7 * 4 / 0.020) < 1e-6          # whole-job events / max time


# ---------------------------------------------------------------- log-det VJP
def _worker_logdet(rank, world, port, out):
    _init(rank, world, port)
    import gwcat
    import oracle
    from tests.helpers import oracle_catalog
    cat, _, _ = oracle_catalog("c4", world, max_npts=60)
    det, psd, rot = gwcat.network("c4")
    g, _ = oracle.logdet_grad_gamma(cat.subset(np.array([rank])), det, psd, rot, 11, [1, 2])
    t = torch.tensor(np.asarray(g), dtype=torch.float64)
    shard.sum_partials(t, world, dist)
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
