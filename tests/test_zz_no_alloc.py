"""gw_fisher_noalloc, the allocation-free Fisher pass, against gw_fisher.

Some callers cannot allocate device memory while they run (code inside a
stream capture that forbids cudaMalloc, applications that reserve all device
memory up front in their own pool, real-time loops).  gw_fisher_noalloc serves
them from a static device array; this test checks, through the C ABI, that two
calls in a row (different catalogs, both precisions) give the results of
gw_fisher, and that a request beyond the static capacity is refused.
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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_gw_fisher_two_calls(prec):
    cases = [_case("c1", 6, 600, 101), _case("c4", 9, None, 202)]
    for gcat, net, P in cases:       # two calls in a row on different catalogs
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


def test_noalloc_refuses_beyond_capacity():
    d = gwcat.draw("c3", 200_000)
    cat = gw.gw_prepare_catalog(d, d["npts_rule"])
    net = gw.Network(*gwcat.network("c3"))
    F = torch.empty((66, cat.n), dtype=torch.float64, device="cuda")
    st = torch.empty(cat.n, dtype=torch.int32, device="cuda")
    assert gw.gw_fisher_noalloc(cat, net, 11, F, None, st, gw.GW_FP64) == gw.GW_ETOOLARGE
