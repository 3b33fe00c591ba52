"""Write tests/golden/parity_oracle.npz: oracle Fisher matrices and SNRs of
stratified subsets of the synthetic catalogs, for the GPU parity tests.

The oracle (``oracle/``, long double, Richardson differences) costs about a
second per 200-point event, too slow to run on a thousand events inside a GPU
test, so its results are stored.  This script calls only ``oracle/`` and the
seeded input generators of ``gwcat``; nothing here comes from the CUDA path.

Sets (every event with its oracle-prepared parameters, grid, Fisher matrix,
SNR, and the oracle's inversion: covariance, condition number, status):
  c3lit  1000 events of the 1e5-event c3 catalog (literal 40-per-e-fold grid),
         stratified by class x grid length: 500 BBH (all 200 points; spread
         over total-mass deciles) and 500 tidal BNS over three grid-length bins
  c3str  160 events of the stress catalog (log-uniform 200..20000 points),
         20 per class x grid-length quarter (in log N)
  long   4 events of the stress catalog with 15000..20000 points
         (2 BBH, 2 BNS): 59..79 work items each
  c4     150 events of the c4 catalog (triangle + two L detectors), 100 BBH
         and 50 BNS

Run:  python tests/golden/make_parity_golden.py   (a few minutes on 8 cores)
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gwcat      # noqa: E402
import oracle     # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "parity_oracle.npz")
SEED = 20221207


def _prepared(cfg, grid):
    """The whole catalog of ``cfg`` prepared by the oracle: event rows [n, 13],
    pset, fmin, fmax (= f_ISCO), npts."""
    d = gwcat.draw(cfg, grid=grid)
    p = oracle.prepare(d["m1"], d["m2"], d["chi1"], d["chi2"], d["lam1"], d["lam2"],
                       d["dL_Mpc"], d["zflag"], d["tcoal"])
    ev = np.stack([p["Mc"], p["eta"], p["dL"], d["theta"], d["phi"], d["iota"], d["psi"],
                   p["tc"], d["Phic"], p["chi1z"], p["chi2z"], p["LamT"], p["dLamT"]], 1)
    rule = d["npts_rule"]
    if rule[0] == "efold":
        npts = oracle.grid_npts(d["fmin"], p["fisco"], *rule[1:])
    else:
        npts = d["npts"].astype(np.int32)
    mtot = d["m1"] + d["m2"]
    return ev, d["pset"], d["fmin"], p["fisco"], npts, mtot


def _pick(rng, idx, k):
    idx = np.asarray(idx)
    return np.sort(rng.choice(idx, min(k, len(idx)), replace=False))


def _strata_c3lit(rng, pset, npts, mtot):
    bbh = np.nonzero(pset == 1)[0]
    bns = np.nonzero(pset == 2)[0]
    out = []
    dec = np.quantile(mtot[bbh], np.linspace(0, 1, 11))
    for a, b in zip(dec[:-1], dec[1:]):
        out.append(_pick(rng, bbh[(mtot[bbh] >= a) & (mtot[bbh] <= b)], 50))
    edges = np.quantile(npts[bns], [0, 1 / 3, 2 / 3, 1])
    for j, (a, b) in enumerate(zip(edges[:-1], edges[1:])):
        m = (npts[bns] >= a) & ((npts[bns] < b) if j < 2 else (npts[bns] <= b))
        out.append(_pick(rng, bns[m], 167 if j < 2 else 166))
    return np.unique(np.concatenate(out))


def _strata_c3str(rng, pset, npts):
    out = []
    edges = np.exp(np.linspace(np.log(200), np.log(20000), 5))
    for cls in (1, 2):
        c = np.nonzero(pset == cls)[0]
        for a, b in zip(edges[:-1], edges[1:]):
            out.append(_pick(rng, c[(npts[c] >= a) & (npts[c] < b + 1)], 20))
    return np.unique(np.concatenate(out))


def _long(rng, pset, npts):
    out = []
    for cls in (1, 2):
        c = np.nonzero((pset == cls) & (npts >= 15000) & (npts <= 20000))[0]
        out.append(_pick(rng, c, 2))
    return np.unique(np.concatenate(out))


def _c4(rng, pset):
    return np.unique(np.concatenate([_pick(rng, np.nonzero(pset == 1)[0], 100),
                                     _pick(rng, np.nonzero(pset == 2)[0], 50)]))


def _one(args):
    ev, pset, fmin, fmax, npts, cfg = args
    det, psd, rot = gwcat.network(cfg)
    cat = oracle.Catalog(ev[None], pset, fmin, fmax, npts)
    F, s, err, st = oracle.fisher(cat, det, psd, rot, 11)
    return F[0], s[0], err[0], st[0]


def main():
    oracle.build()
    rng = np.random.default_rng(SEED)
    sets = {}
    ev, pset, fmin, fmax, npts, mtot = _prepared("c3", "literal")
    sets["c3lit"] = ("c3", _strata_c3lit(rng, pset, npts, mtot), ev, pset, fmin, fmax, npts)
    ev, pset, fmin, fmax, npts, mtot = _prepared("c3", "stress")
    sets["c3str"] = ("c3", _strata_c3str(rng, pset, npts), ev, pset, fmin, fmax, npts)
    sets["long"] = ("c3", _long(rng, pset, npts), ev, pset, fmin, fmax, npts)
    ev, pset, fmin, fmax, npts, mtot = _prepared("c4", "literal")
    sets["c4"] = ("c4", _c4(rng, pset), ev, pset, fmin, fmax, npts)

    out = {}
    iu = np.triu_indices(11)
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        for name, (cfg, idx, ev, pset, fmin, fmax, npts) in sets.items():
            t0 = time.time()
            # longest events first so that the pool stays busy
            order = idx[np.argsort(-npts[idx], kind="stable")]
            res = pool.map(_one, [(ev[i], pset[i], fmin[i], fmax[i], npts[i], cfg)
                                  for i in order], chunksize=1)
            back = np.argsort(np.argsort(-npts[idx], kind="stable"), kind="stable")
            res = [res[k] for k in back]
            F = np.array([r[0] for r in res])
            out[f"{name}_config"] = np.array(cfg)
            out[f"{name}_row"] = idx.astype(np.int64)
            out[f"{name}_ev"] = ev[idx]
            out[f"{name}_pset"] = pset[idx]
            out[f"{name}_fmin"] = fmin[idx]
            out[f"{name}_fmax"] = fmax[idx]
            out[f"{name}_npts"] = npts[idx]
            out[f"{name}_fisher"] = F[:, iu[0], iu[1]]        # packed upper, row-major
            out[f"{name}_snr"] = np.array([r[1] for r in res])
            out[f"{name}_fd_err"] = np.array([r[2] for r in res])
            out[f"{name}_status"] = np.array([r[3] for r in res], dtype=np.int32)
            # the oracle's long-double inversion of its own Fisher matrices (Sec. 4.1)
            C, kappa, inv_err, inv_st = oracle.invert(F)
            out[f"{name}_cov"] = C[:, iu[0], iu[1]]
            out[f"{name}_kappa"] = kappa
            out[f"{name}_inv_status"] = inv_st.astype(np.int32)
            print(f"{name}: {len(idx)} events, {int(npts[idx].sum())} points, "
                  f"{time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
