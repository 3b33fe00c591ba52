"""gw_fisher_refine: events of a mixed pass whose inversion fails or whose
condition number exceeds the threshold get the FP64 path's results, bit for
bit; every other event keeps its mixed results untouched.  Checked on a
300-event c3 catalog, directly and through a row selection of the catalog."""
import numpy as np
import pytest
import torch

import gwcat
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def _pass(cat, net, prec, up):
    F, snr, st, g = gw.gw_fisher(cat, net, 11, prec, grad_snr=up)
    inv = gw.gw_fisher_inverse(F, 11)
    return [F, snr, st, g, *inv]


@pytest.mark.parametrize("selected", [False, True])
def test_refine_is_fp64_on_the_refined_events(selected):
    cat, d, p = oracle_catalog("c3", 300)
    net = gw.Network(*gwcat.network("c3"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    if selected:   # every other row, in reverse order
        gcat = gcat.select(torch.arange(298, -1, -2, device="cuda"))
    up = torch.linspace(0.5, 2.0, gcat.n, dtype=torch.float64, device="cuda")
    mixed = _pass(gcat, net, gw.GW_MIXED, up)
    ref64 = _pass(gcat, net, gw.GW_FP64, up)
    before = [t.clone() for t in mixed]
    F, snr, st, g, cov, cond, err, sti = mixed
    refined = torch.zeros(gcat.n, dtype=torch.uint8, device="cuda")
    n_ref = gw.gw_fisher_refine(gcat, net, 11, F, snr, st, (cov, cond, err, sti), grad_snr=up,
                                grad_params=g, refined=refined)
    torch.cuda.synchronize()
    r = refined.bool()
    want = (before[2] == 0) & (((before[7] & (gw.ST_NOT_PD | gw.ST_NONFINITE)) != 0) |
                               ~(before[5] <= gw.REFINE_COND))
    assert torch.equal(r, want) and n_ref == int(r.sum()) and 0 < n_ref < gcat.n
    for got, old, fp64 in zip(mixed, before, ref64):
        cols = (slice(None), r) if got.dim() == 2 else (r,)
        keep = (slice(None), ~r) if got.dim() == 2 else (~r,)
        assert torch.equal(got[cols].nan_to_num(7.0), fp64[cols].nan_to_num(7.0))
        assert torch.equal(got[keep].nan_to_num(7.0), old[keep].nan_to_num(7.0))


def test_refine_thresholds_and_empty():
    cat, d, p = oracle_catalog("c3", 40)
    net = gw.Network(*gwcat.network("c3"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_MIXED)
    inv = gw.gw_fisher_inverse(F, 11)
    # threshold 0: every clean event is refined; the result is the FP64 pass
    n0 = gw.gw_fisher_refine(gcat, net, 11, F, snr, st, inv, cond_th=0.0)
    F64, s64, st64 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
    assert n0 == gcat.n and torch.equal(F, F64) and torch.equal(snr, s64)
    # an infinite threshold refines only events whose inversion failed
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_MIXED)
    inv = gw.gw_fisher_inverse(F, 11)
    failed = int(((inv[3] & (gw.ST_NOT_PD | gw.ST_NONFINITE)) != 0).sum())
    assert gw.gw_fisher_refine(gcat, net, 11, F, snr, st, inv, cond_th=float("inf")) == failed
    empty = gcat.select(torch.empty(0, dtype=torch.int64, device="cuda"))
    assert gw.gw_fisher_refine(empty, net, 11, F[:, :0], snr[:0], st[:0],
                               tuple(t[..., :0] for t in inv)) == 0
    with pytest.raises(gw.GWError):
        gw.gw_fisher_refine(gcat, net, 11, F, snr, st, inv, cond_th=float("nan"))
