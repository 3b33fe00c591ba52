"""Run oracle calls for many events in a spawn process pool (one event per
task), so the parity tests finish in bounded time on a many-core host.  The
pool uses the 'spawn' start method: a pool forked after CUDA is initialised in
the parent can hang."""
import multiprocessing as mp
import os

import numpy as np

_POOL = None


def _worker_fisher(args):
    import oracle
    ev, pset, fmin, fmax, npts, mask, det, psd, rot, n_par = args[:10]
    if len(args) > 10:            # tabulated PSDs of this network
        oracle.set_psd_tables(args[10])
    cat = oracle.Catalog(ev, pset, fmin, fmax, npts, mask)
    F, s, err, st = oracle.fisher(cat, det, psd, rot, n_par)
    return F[0], s[0], err[0], st[0]


def _worker_snr(args):
    import oracle
    ev, pset, fmin, fmax, npts, mask, det, psd, rot = args[:9]
    if len(args) > 9:
        oracle.set_psd_tables(args[9])
    cat = oracle.Catalog(ev, pset, fmin, fmax, npts, mask)
    s, arm, st = oracle.snr(cat, det, psd, rot, per_arm=True)
    return s[0], arm[0], st[0]


def _worker_grad(args):
    import oracle
    ev, pset, fmin, fmax, npts, mask, det, psd, rot, n_par = args
    cat = oracle.Catalog(ev, pset, fmin, fmax, npts, mask)
    return oracle.snr_grad(cat, det, psd, rot, n_par)[0]


def _worker_logdet(args):
    import oracle
    ev, pset, fmin, fmax, npts, mask, det, psd, rot, n_par, dets = args
    cat = oracle.Catalog(ev, pset, fmin, fmax, npts, mask)
    g, ld = oracle.logdet_grad_gamma(cat, det, psd, rot, n_par, dets)
    return g, ld[0]


def pool():
    global _POOL
    if _POOL is None:
        import oracle
        oracle.build()
        _POOL = mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))
    return _POOL


def _tasks(cat, extra):
    return [(cat.ev[e], cat.pset[e], cat.fmin[e], cat.fmax[e], cat.npts[e],
             None if cat.arm_mask is None else cat.arm_mask[e], *extra)
            for e in range(len(cat))]


def fisher(cat, det, psd, rot, n_par, tables=None):
    extra = (det, psd, rot, n_par) + ((tables,) if tables is not None else ())
    out = pool().map(_worker_fisher, _tasks(cat, extra))
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]), np.array([o[3] for o in out]))


def snr(cat, det, psd, rot, tables=None):
    extra = (det, psd, rot) + ((tables,) if tables is not None else ())
    out = pool().map(_worker_snr, _tasks(cat, extra))
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]))


def snr_grad(cat, det, psd, rot, n_par):
    return np.array(pool().map(_worker_grad, _tasks(cat, (det, psd, rot, n_par))))


def logdet_grad(cat, det, psd, rot, n_par, dets):
    out = pool().map(_worker_logdet, _tasks(cat, (det, psd, rot, n_par, list(dets))))
    return np.sum([o[0] for o in out], axis=0), np.array([o[1] for o in out])
