"""gw_fisher_noalloc, the allocation-free Fisher pass, against gw_fisher.

Some callers must not allocate device memory while they run: an application
that hands all device memory to its own fixed-size pool at start-up, or a
long-running loop that cannot afford an allocation's latency, implicit
synchronisation or failure halfway through a job.  gw_fisher_noalloc serves
them from a static device array.  These tests check, through the C ABI, that
two calls in a row (different catalogs, both precisions) give the results of
gw_fisher, that the documented size (1e4 events of 512 points on a triangle)
fits, and that requests beyond the static capacity are refused, before and
after the work-item count is known, without touching the outputs.
The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import gwcat
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def _case(cfg, n, cap, seed):
    cat, d, p = oracle_catalog(cfg, n, max_npts=cap, seed=seed)
    det, psd, rot = gwcat.network(cfg)
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    return gcat, gw.Network(det, psd, rot), gwcat.N_PAR[cfg]


def _check_against_gw_fisher(gcat, net, P, prec):
    F_ref, s_ref, st_ref = gw.gw_fisher(gcat, net, P, prec)
    F = torch.full_like(F_ref, np.nan)
    s = torch.full_like(s_ref, np.nan)
    st = torch.full_like(st_ref, -1)
    assert gw.gw_fisher_noalloc(gcat, net, P, F, s, st, prec) == 0
    torch.cuda.synchronize()
    assert torch.equal(st, st_ref) and int((st != 0).sum()) == 0
    Fr = gw.unpack(F_ref, P).cpu().numpy()
    Fn = gw.unpack(F, P).cpu().numpy()
    dg = np.sqrt(np.einsum("eii->ei", Fr))
    rel = np.abs(Fn - Fr) / (dg[:, :, None] * dg[:, None, :])
    tol_f, tol_s = (1e-8, 1e-10) if prec == 0 else (2e-6, 1e-5)
    assert rel.max() < tol_f
    assert torch.max(torch.abs(s / s_ref - 1)).item() < tol_s


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_gw_fisher_two_calls(prec):
    cases = [_case("c1", 6, 600, 101), _case("c4", 9, None, 202)]
    for gcat, net, P in cases:       # two calls in a row on different catalogs
        _check_against_gw_fisher(gcat, net, P, prec)


def test_noalloc_documented_size_fits():
    """1e4 events of 512 grid points each on one triangle (the size the header
    names) fit the static workspace in the mixed path, the larger of the two."""
    d = gwcat.draw("c3", 10_000)
    d["npts"] = np.full(10_000, 512, dtype=np.int32)
    cat = gw.gw_prepare_catalog(d, ("given",))
    net = gw.Network(*gwcat.network("c3"))
    _check_against_gw_fisher(cat, net, 11, gw.GW_MIXED)


def test_noalloc_refuses_beyond_capacity():
    # too many events: refused before any launch (event constants alone overflow)
    d = gwcat.draw("c3", 200_000)
    cat = gw.gw_prepare_catalog(d, d["npts_rule"])
    net = gw.Network(*gwcat.network("c3"))
    F = torch.full((66, cat.n), 7.0, dtype=torch.float64, device="cuda")
    st = torch.empty(cat.n, dtype=torch.int32, device="cuda")
    assert gw.gw_fisher_noalloc(cat, net, 11, F, None, st, gw.GW_FP64) == gw.GW_ETOOLARGE
    assert bool(torch.all(F == 7.0))
    # few events with long grids: the event constants fit, the per-item partial
    # sums do not; refused after the work-item scan, outputs untouched
    d = gwcat.draw("c3", 3000)
    d["npts"] = np.full(3000, 8000, dtype=np.int32)
    cat = gw.gw_prepare_catalog(d, ("given",))
    F = torch.full((66, cat.n), 7.0, dtype=torch.float64, device="cuda")
    s = torch.full((cat.n,), 7.0, dtype=torch.float64, device="cuda")
    st = torch.empty(cat.n, dtype=torch.int32, device="cuda")
    assert gw.gw_fisher_noalloc(cat, net, 11, F, s, st, gw.GW_FP64) == gw.GW_ETOOLARGE
    torch.cuda.synchronize()
    assert bool(torch.all(F == 7.0)) and bool(torch.all(s == 7.0))
    # and a call that fits still works after the refusals
    gcat, net2, P = _case("c1", 5, 700, 303)
    _check_against_gw_fisher(gcat, net2, P, gw.GW_MIXED)
