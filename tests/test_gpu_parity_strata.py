"""Parity of the CUDA path with the oracle on stratified catalog subsets.

The oracle's Fisher matrices and SNRs of 1000 events of the c3 catalog
(literal grid; 500 BBH over total-mass deciles, 500 tidal BNS over three
grid-length bins), 160 events of the stress catalog (class x grid-length
quarter), four 15000..20000-point events (59..79 work items each) and 150 events
of the five-interferometer c4 catalog are stored in tests/golden/parity_oracle.npz
(written by tests/golden/make_parity_golden.py, which calls only the oracle).
The covariances of reference are the oracle's long-double inversion of its own
Fisher matrices (Sec. 4.1).

Arms: the FP64 path with its Gram on the FP64 pipe and on the tensor cores
(exact digit products); the double-float path (GW_DFLOAT: every per-point
quantity in double-float on the FP32 pipe, the Gram exact on the tensor cores;
the c4 network, four interferometers per point, runs it as FP64); the mixed
path alone; the mixed path followed by gw_fisher_refine (events whose mixed
inversion fails or whose condition number exceeds 1e7 recomputed in FP64),
which is the mixed path's result of record; and the routed step
(gw_fisher_routed: the BBH by the double-float pass, the BNS by the mixed
pass, those failing the same check recomputed by the double-float pass).

Tolerances, per event:
  SNR                FP64 and double-float 1e-10 relative, mixed 1e-5; the
                     routed step's BBH the former, its BNS the latter.
  Gamma_ij           FP64 and double-float 1e-8 of sqrt(Gamma_ii Gamma_jj),
                     mixed 2e-6 (routed: as for SNR).
  sqrt(diag C)       1e-3 relative, or the FP64 floor B * kappa where that is
                     larger (FP64, double-float, refined mixed and routed arms).  kappa is the
                     oracle's 2-norm condition number of the normalised Fisher
                     matrix.  Both Fisher matrices are FP64 arrays: rounding
                     each element of Gamma to FP64 (u = 2^-53, P = 11) moves
                     sqrt(diag C) by up to ~P u kappa = 1.2e-15 kappa, so above
                     kappa ~ 1e12 no FP64 Fisher matrix, the oracle's included,
                     fixes sqrt(diag C) to 1e-3.  B = 1e-15 (measured: at most
                     3e-16 kappa).  The mixed arm alone is held to 1e-3 on the
                     events gw_fisher_refine keeps (GPU condition number <= 1e7);
                     its error on the others (~1e-13 kappa) is printed.
  Events the oracle's inversion flags NOT_PD or ILL_COND (kappa above 1/eps,
  the paper's limit of a reliable inversion) are left out of the covariance
  check and counted.  A per-decade table of the strict 1e-3 pass fraction is
  printed for every set and arm.
"""
import math
import os

import numpy as np
import pytest
import torch

import gwcat
import oracle

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "parity_oracle.npz")
SETS = ("c3lit", "c3str", "long", "c4")
ARMS = ("fp64", "fp64_tc", "dfloat", "mixed", "mixed_refined", "routed")
B_COV = 1e-15
TOL_SNR = {"fp64": 1e-10, "fp64_tc": 1e-10, "dfloat": 1e-10, "mixed": 1e-5, "mixed_refined": 1e-5}
TOL_F = {"fp64": 1e-8, "fp64_tc": 1e-8, "dfloat": 1e-8, "mixed": 2e-6, "mixed_refined": 2e-6}
ROUTED_PSETS = 1 << 1          # the BBH to the double-float pass


def _tol(tol, arm, pset):
    """Per-event tolerance: the routed step's events by the pass they were
    routed to (the mixed ones may have been recomputed: the looser bound)."""
    if arm != "routed":
        return tol[arm]
    return np.where((ROUTED_PSETS >> pset.astype(np.int64)) & 1 == 1, tol["dfloat"], tol["mixed"])


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.fail("tests/golden/parity_oracle.npz is missing: run tests/golden/make_parity_golden.py")
    z = np.load(GOLDEN)
    out = {}
    iu = np.triu_indices(11)
    for s in SETS:
        Fp = z[f"{s}_fisher"]
        F = np.zeros((len(Fp), 11, 11))
        F[:, iu[0], iu[1]] = Fp
        F[:, iu[1], iu[0]] = Fp
        C, kappa, eps, st = oracle.invert(F)
        out[s] = dict(cfg=str(z[f"{s}_config"]), ev=z[f"{s}_ev"], pset=z[f"{s}_pset"],
                      fmin=z[f"{s}_fmin"], fmax=z[f"{s}_fmax"], npts=z[f"{s}_npts"],
                      F=F, snr=z[f"{s}_snr"], ost=z[f"{s}_status"], C=C, kappa=kappa, inv_st=st)
    return out


def _run(r, arm):
    det, psd, rot = gwcat.network(r["cfg"])
    net = gw.Network(det, psd, rot)
    cat = gw.Catalog.from_numpy(r["ev"], r["pset"], r["fmin"], r["fmax"], r["npts"])
    if arm == "routed":
        F, snr, st, C, cond, err, sti, n_df, n_ref = gw.gw_fisher_routed(cat, net, 11, ROUTED_PSETS)
        assert n_df == int(np.sum((ROUTED_PSETS >> r["pset"].astype(np.int64)) & 1))
        torch.cuda.synchronize()
        return (gw.unpack(F, 11).cpu().numpy(), snr.cpu().numpy(), st.cpu().numpy(),
                gw.unpack(C, 11).cpu().numpy(), cond.cpu().numpy(), sti.cpu().numpy(), n_ref)
    prec = {"fp64": gw.GW_FP64, "fp64_tc": gw.GW_FP64, "dfloat": gw.GW_DFLOAT}.get(arm, gw.GW_MIXED)
    gw.gw_set_fp64_gram(arm == "fp64_tc")
    try:
        F, snr, st = gw.gw_fisher(cat, net, 11, prec)
    finally:
        gw.gw_set_fp64_gram(False)
    inv = gw.gw_fisher_inverse(F, 11)
    n_ref = 0
    if arm == "mixed_refined":
        n_ref = gw.gw_fisher_refine(cat, net, 11, F, snr, st, inv)
    C, cond, err, sti = inv
    torch.cuda.synchronize()
    return (gw.unpack(F, 11).cpu().numpy(), snr.cpu().numpy(), st.cpu().numpy(),
            gw.unpack(C, 11).cpu().numpy(), cond.cpu().numpy(), sti.cpu().numpy(), n_ref)


def decade_table(kappa, rel, ok, tol=1e-3):
    """Rows (decade, events, strict pass fraction, median, max) of the relative
    sqrt(diag C) error over the oracle's condition-number decades."""
    rows = []
    dec = np.floor(np.log10(np.maximum(kappa, 1.0))).astype(int)
    for d in range(dec.min(), dec.max() + 1):
        m = ok & (dec == d)
        if m.any():
            rows.append((d, int(m.sum()), float(np.mean(rel[m] <= tol)), float(np.median(rel[m])),
                         float(np.max(rel[m]))))
    return rows


@pytest.mark.parametrize("arm", ARMS)
@pytest.mark.parametrize("name", SETS)
def test_strata_against_oracle(golden, name, arm):
    r = golden[name]
    F, snr, st, C, cond, sti, n_ref = _run(r, arm)
    n = len(snr)
    assert np.all(r["ost"] == 0) and np.all(st == 0)
    # SNR and Fisher matrix, every event
    assert np.all(np.abs(snr / r["snr"] - 1) < _tol(TOL_SNR, arm, r["pset"]))
    dg = np.sqrt(np.einsum("eii->ei", r["F"]))
    relF = np.abs(F - r["F"]) / (dg[:, :, None] * dg[:, None, :])
    worstF = relF.reshape(n, -1).max(1)
    badF = ~(worstF < _tol(TOL_F, arm, r["pset"]))
    assert not badF.any(), (worstF.max(), int(worstF.argmax()))
    # marginalised errors sqrt(diag C)
    kappa = r["kappa"]
    flagged = (r["inv_st"] & (oracle.ST_NOT_PD | oracle.ST_ILL_COND)) != 0
    gpu_notpd = (sti & gw.ST_NOT_PD) != 0
    ok = ~flagged & ~gpu_notpd
    so = np.sqrt(np.abs(np.einsum("eii->ei", r["C"])))
    sg = np.sqrt(np.abs(np.einsum("eii->ei", C)))
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.max(np.abs(sg / so - 1), axis=1)
    rows = decade_table(kappa, rel, ok)
    how = "recomputed in double-float" if arm == "routed" else "refined in FP64"
    print(f"\n{name} {arm}: {n} events, {n_ref} {how}, {int(flagged.sum())} flagged by "
          f"the oracle (NOT_PD/ILL_COND), {int((gpu_notpd & ~flagged).sum())} more NOT_PD on the GPU")
    print(" kappa decade  events  pass(1e-3)  median rel  max rel")
    for d, k, f, med, mx in rows:
        print(f"   1e{d:<3d}      {k:6d}   {f:8.3f}   {med:9.2e}  {mx:9.2e}")
    if arm == "mixed":
        check = ok & (cond <= gw.REFINE_COND)
        bound = np.full(n, 1e-3)
    else:
        check = ok
        bound = np.maximum(1e-3, B_COV * kappa)
    bad = check & ~(rel <= bound)
    assert not bad.any(), [(int(e), float(rel[e]), float(kappa[e])) for e in np.nonzero(bad)[0][:8]]
    if arm != "mixed":
        # an event the GPU cannot factorise must be one beyond the FP64 floor
        assert np.all(kappa[gpu_notpd & ~flagged] > 1e13), kappa[gpu_notpd & ~flagged]
