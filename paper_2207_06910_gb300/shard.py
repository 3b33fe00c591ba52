"""Splitting one catalog over several processes (one per GPU) and gathering the
per-event results back in catalog order.

The paper's forecast driver splits a catalog into index ranges ([idx_in, idx_f)
of Sec. 5) and hands batches to a pool of processes or MPI ranks.  Events are
independent, so no exchange is needed for SNR, Fisher matrices, covariances or
the SNR VJP; the only cross-event quantity, the log-det VJP, is a sum of
per-shard partial sums.  Here the split is into contiguous ranges whose costs
are balanced: an event costs its grid points times its number of effective
interferometers (a triangle with all arms on counts two, see the point
kernels), the work of the fused point loop.  This module is host logic only
(numpy and torch.distributed): no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np


def event_cost(npts, d_eff) -> np.ndarray:
    """Cost of each event: grid points x effective interferometers."""
    npts = np.asarray(npts, dtype=np.float64)
    return npts * np.broadcast_to(np.asarray(d_eff, dtype=np.float64), npts.shape)


def partition(cost, world: int) -> np.ndarray:
    """Boundaries b[0] = 0 <= b[1] <= ... <= b[world] = n of ``world``
    contiguous ranges [b[r], b[r+1]) of the events whose summed costs are as
    equal as contiguous ranges allow: boundary r sits where the running cost
    is nearest to r / world of the total, so every range's cost differs from
    total / world by at most the cost of one event (half an event at each end)."""
    cost = np.asarray(cost, dtype=np.float64)
    n = len(cost)
    if world < 1:
        raise ValueError("world must be >= 1")
    if np.any(cost < 0) or not np.all(np.isfinite(cost)):
        raise ValueError("costs must be finite and >= 0")
    cum = np.concatenate([[0.0], np.cumsum(cost)])      # cum[k] = cost of events < k
    total = cum[-1]
    b = np.empty(world + 1, dtype=np.int64)
    b[0], b[world] = 0, n
    for r in range(1, world):
        t = total * r / world
        k = int(np.searchsorted(cum, t))                 # cum[k-1] < t <= cum[k]
        if k > 0 and (k > n or t - cum[k - 1] < cum[k] - t):
            k -= 1
        b[r] = min(max(k, b[r - 1]), n)
    return b


def my_range(cost, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's events."""
    b = partition(cost, world)
    return int(b[rank]), int(b[rank + 1])


def imbalance(cost, bounds) -> float:
    """max over ranges of |range cost - total / world|."""
    cost = np.asarray(cost, dtype=np.float64)
    world = len(bounds) - 1
    total = float(cost.sum())
    return max(abs(float(cost[bounds[r]:bounds[r + 1]].sum()) - total / world)
               for r in range(world))


def gather_events(local, bounds, rank: int, world: int, dist=None, dst: int = 0):
    """Concatenate, in catalog order, every rank's per-event result arrays.

    ``local`` is a dict of arrays (numpy or torch CPU) whose LAST axis is the
    rank's events ([..., n_rank], the event-minor layout of the library's
    outputs).  With world = 1 (or no process group) it is returned as is.
    Otherwise every rank sends its arrays to ``dst`` (torch.distributed
    gather_object, any backend); ``dst`` returns the concatenated dict, the
    other ranks None."""
    if world == 1 or dist is None:
        return {k: np.asarray(v) for k, v in local.items()}
    n_r = int(bounds[rank + 1] - bounds[rank])
    payload = {k: np.asarray(v.cpu() if hasattr(v, "cpu") else v) for k, v in local.items()}
    for k, v in payload.items():
        if v.shape[-1] != n_r:
            raise ValueError(f"{k}: last axis {v.shape[-1]} != the rank's {n_r} events")
    out = [None] * world if rank == dst else None
    dist.gather_object((rank, payload), out, dst=dst)
    if rank != dst:
        return None
    parts = sorted(out, key=lambda x: x[0])
    return {k: np.concatenate([p[1][k] for p in parts], axis=-1) for k in local}


def sum_partials(t, world: int, dist=None):
    """Whole-catalog value of a per-shard partial sum (the log-det gradient),
    in place: all-reduce SUM over the ranks; a no-op on one rank."""
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
