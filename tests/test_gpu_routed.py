"""gw_fisher_routed: the Fisher pass and inversion with the precision chosen per
event, against the passes it routes to.

Events of the parameter sets named by dfloat_psets (here the BBH, pset 1)
run the double-float pass, the others the mixed pass; mixed events whose
inversion failed or whose condition number exceeds cond_th are recomputed by
the double-float pass (Sec. 4.1's conditioning check applied to the Fisher
matrix's precision).  An event's results depend only on its own work items,
so the routed results equal, bit for bit, those of the double-float pass +
inversion for the routed and the recomputed events and of the mixed pass +
inversion for the others, with the fused SNR VJP scattered the same way."""
import numpy as np
import pytest
import torch

import gwcat
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def _full(gcat, net, prec, up):
    F, snr, st, g = gw.gw_fisher(gcat, net, 11, prec, grad_snr=up)
    inv = gw.gw_fisher_inverse(F, 11)
    return F, snr, st, g, inv


@pytest.mark.parametrize("mask", [1 << 1, 0, (1 << 1) | (1 << 2)])
def test_routed_equals_its_passes(mask):
    cat, d, p = oracle_catalog("c3", 60, seed=20220714 + 46)
    net = gw.Network(*gwcat.network("c3"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    up = torch.linspace(0.5, 1.5, 60, dtype=torch.float64, device="cuda")
    out = gw.gw_fisher_routed(gcat, net, 11, mask, grad_snr=up)
    F, snr, st, cov, cond, err, sti, g, n_df, n_ref = out
    pset = np.asarray(cat.pset)
    to_df = np.array([(mask >> int(ps)) & 1 for ps in pset], dtype=bool)
    assert n_df == int(to_df.sum())
    D = _full(gcat, net, gw.GW_DFLOAT, up)
    M = _full(gcat, net, gw.GW_MIXED, up)
    # the refinement's rule on the mixed results: a clean point-loop status and a
    # failed inversion (NOT_PD, NONFINITE) or a condition number above 1e7
    cond_m, sti_m = M[4][1], M[4][3]
    redo = (M[2] == 0) & (((sti_m & 5) != 0) | ~(cond_m <= gw.REFINE_COND))
    sel_df = torch.as_tensor(to_df, device="cuda")
    assert n_ref == int((redo & ~sel_df).sum())
    sel_df = sel_df | redo
    for k, (got, a, b) in enumerate(((F, D[0], M[0]), (snr, D[1], M[1]), (st, D[2], M[2]),
                                     (g, D[3], M[3]), (cov, D[4][0], M[4][0]),
                                     (cond, D[4][1], M[4][1]), (err, D[4][2], M[4][2]),
                                     (sti, D[4][3], M[4][3]))):
        want = torch.where(sel_df, a, b)
        assert torch.equal(got, want), k
    assert int((st != 0).sum()) == 0
    if mask == 0:
        assert n_df == 0 and n_ref > 0        # every event mixed: the BBH get refined
    assert gw.gw_kernel_faults() == 0


def test_routed_sqrt_diag_cov_tolerance():
    """The routed step's marginalised errors against the double-float ones: the
    mixed events (BNS here, well conditioned, or refined) within 1e-3."""
    cat, d, p = oracle_catalog("c3", 80, seed=20220714 + 47)
    net = gw.Network(*gwcat.network("c3"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    F, snr, st, cov, cond, err, sti, n_df, n_ref = gw.gw_fisher_routed(gcat, net, 11, 1 << 1)
    Fd, sd, std_ = gw.gw_fisher(gcat, net, 11, gw.GW_DFLOAT)
    covd = gw.gw_fisher_inverse(Fd, 11)[0]
    ok = ((sti == 0) & (gw.gw_fisher_inverse(Fd, 11)[3] == 0)).cpu().numpy()
    a = np.sqrt(np.abs(np.einsum("eii->ei", gw.unpack(cov, 11).cpu().numpy())))[ok]
    b = np.sqrt(np.abs(np.einsum("eii->ei", gw.unpack(covd, 11).cpu().numpy())))[ok]
    assert ok.sum() > 40
    assert np.max(np.abs(a / b - 1)) < 1e-3
    assert np.max(np.abs(snr.cpu().numpy() / sd.cpu().numpy() - 1)) < 1e-5
