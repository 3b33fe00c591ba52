"""GW_DFLOAT: the Fisher pass with every per-point quantity in double-float
arithmetic on the FP32 pipe and the Gram of the tangents exact on the tensor
cores, against the FP64 pass and the oracle.

The two paths evaluate the same formulas (Sec. 3.2, Eqs. 3.1-3.3; one templated
source) in FP64 and in double-float (~2^-48 per operation): the tangents agree
to ~1e-14 relative, so the Fisher matrices agree to ~1e-13 of
sqrt(Gamma_ii Gamma_jj) (bound 1e-10) and the SNRs to ~1e-14 (bound 1e-12).
Against the oracle the FP64 bounds apply (Gamma_ij 1e-8, SNR 1e-10).  The
covariance accuracy over the condition-number decades is checked on the 1000
stratified events in test_gpu_parity_strata.py.

Cases: one- and two-round work items, both parameter counts (9: one L-shaped
detector, no Earth rotation; 11: the rotating triangle), long grids, a
tabulated PSD (its weight taken in FP64), duty-factor arm masks, and a network
of four interferometers per point (not supported by the tensor-core kernel:
GW_DFLOAT then runs the FP64 pass, bit for bit)."""
import numpy as np
import pytest
import torch

import gwcat
from tests import oracle_pool
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def _rel(F1, F2, np_):
    A = gw.unpack(F1, np_).cpu().numpy()
    B = gw.unpack(F2, np_).cpu().numpy()
    dg = np.sqrt(np.abs(np.einsum("eii->ei", B)))
    return float(np.max(np.abs(A - B) / (dg[:, :, None] * dg[:, None, :])))


CASES = {
    "c3_literal": ("c3", 80, "literal", None, 11),
    "c3_stress": ("c3", 12, "stress", None, 11),
    "c1_long": ("c1", 4, "literal", None, 11),
    "c2_bns": ("c2", 6, "literal", 3000, 11),
    "c0_L_norot": ("c0", 20, "literal", None, 9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_dfloat_matches_fp64(name):
    cfg, n, grid, cap, np_ = CASES[name]
    cat, d, p = oracle_catalog(cfg, n, grid=grid, max_npts=cap)
    net = gw.Network(*gwcat.network(cfg))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    up = torch.linspace(0.5, 1.5, n, dtype=torch.float64, device="cuda")
    F1, s1, st1, g1 = gw.gw_fisher(gcat, net, np_, gw.GW_DFLOAT, grad_snr=up)
    F2, s2, st2, g2 = gw.gw_fisher(gcat, net, np_, gw.GW_FP64, grad_snr=up)
    assert torch.equal(st1, st2) and int((st1 != 0).sum()) == 0
    r = _rel(F1, F2, np_)
    rs = torch.max(torch.abs(s1 / s2 - 1)).item()
    print(f"\n{name}: max |dGamma| / sqrt(Gii Gjj) = {r:.2e}, SNR {rs:.2e}")
    assert r < 1e-10
    assert rs < 1e-12
    dgj = torch.sqrt(torch.stack([F2[j * np_ - j * (j - 1) // 2] for j in range(np_)]))
    assert torch.max(torch.abs(g1 - g2) / (dgj * up)).item() < 1e-10
    assert gw.gw_kernel_faults() == 0


def test_dfloat_item_split_edges():
    """Grid lengths around the tensor-core pass's work-item shapes: an event's
    ceil(N/128) items take the even share rounded up to whole warps (32 points),
    the last item the rest.  Lengths at and next to the warp and item edges,
    on the rotating triangle (11 parameters) and one L-shaped detector
    without rotation (9 parameters), against the FP64 pass."""
    lens = [2, 3, 31, 32, 33, 95, 96, 97, 127, 128, 129, 160, 200, 255, 256, 257,
            288, 289, 384, 385, 513]
    for cfg, np_ in (("c3", 11), ("c0", 9)):
        cat, d, p = oracle_catalog(cfg, len(lens), seed=20220714 + 45)
        npts = np.array(lens, dtype=np.int32)
        gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, npts)
        net = gw.Network(*gwcat.network(cfg))
        F1, s1, st1 = gw.gw_fisher(gcat, net, np_, gw.GW_DFLOAT)
        F2, s2, st2 = gw.gw_fisher(gcat, net, np_, gw.GW_FP64)
        assert torch.equal(st1, st2)
        ok = (st1 == 0).cpu().numpy()
        assert ok.sum() >= len(lens) - 2          # (N = 2, 3 may be degenerate)
        F1n, F2n = F1.cpu().numpy()[:, ok], F2.cpu().numpy()[:, ok]
        r = _rel(torch.as_tensor(F1n), torch.as_tensor(F2n), np_)
        rs = float(np.max(np.abs(s1.cpu().numpy()[ok] / s2.cpu().numpy()[ok] - 1)))
        print(f"\n{cfg} split edges: max |dGamma| / sqrt(Gii Gjj) = {r:.2e}, SNR {rs:.2e}")
        assert r < 1e-10 and rs < 1e-12
    assert gw.gw_kernel_faults() == 0


def test_dfloat_against_oracle():
    cat, d, p = oracle_catalog("c3", 24, seed=20220714 + 43)
    det, psd, rot = gwcat.network("c3")
    F_or, s_or, _, st_or = oracle_pool.fisher(cat, det, psd, rot, 11)
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    F, snr, st = gw.gw_fisher(gcat, gw.Network(det, psd, rot), 11, gw.GW_DFLOAT)
    assert int((st != 0).sum()) == 0 and np.all(st_or == 0)
    A = gw.unpack(F, 11).cpu().numpy()
    dg = np.sqrt(np.einsum("eii->ei", F_or))
    rel = np.abs(A - F_or) / (dg[:, :, None] * dg[:, None, :])
    print(f"\nagainst the oracle: max |dGamma| / sqrt(Gii Gjj) = {rel.max():.2e}")
    assert rel.max() < 1e-8
    assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < 1e-10


def test_dfloat_tabulated_psd_and_arm_masks():
    cat, d, p = oracle_catalog("c3", 30, seed=20220714 + 44)
    masks = gwcat.draw_arm_masks(30, 3, 0.7, seed=10)
    det, rows, rot, tables = gwcat.network_tabulated("c3")
    for net, am in ((gw.Network(det, rows, rot, tables), None),
                    (gw.Network(*gwcat.network("c3")), masks)):
        gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, arm_mask=am)
        F1, s1, st1 = gw.gw_fisher(gcat, net, 11, gw.GW_DFLOAT)
        F2, s2, st2 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
        assert torch.equal(st1, st2)
        ok = (st1 == 0).cpu().numpy()
        assert ok.sum() > 10
        F1n, F2n = F1.cpu().numpy()[:, ok], F2.cpu().numpy()[:, ok]
        live = F2n[0] > 0
        assert _rel(torch.as_tensor(F1n[:, live]), torch.as_tensor(F2n[:, live]), 11) < 1e-10
        assert np.all(F1n[:, ~live] == 0)
    assert gw.gw_kernel_faults() == 0


def test_dfloat_wider_network_runs_fp64():
    cat, d, p = oracle_catalog("c4", 8, max_npts=600)
    net = gw.Network(*gwcat.network("c4"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    F1, s1, st1 = gw.gw_fisher(gcat, net, 11, gw.GW_DFLOAT)
    F2, s2, st2 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
    assert torch.equal(F1, F2) and torch.equal(s1, s2)


def test_dfloat_other_passes_are_fp64():
    """The SNR pass at GW_DFLOAT is the FP64 pass (identical bits)."""
    cat, d, p = oracle_catalog("c3", 10)
    net = gw.Network(*gwcat.network("c3"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    a, sa = gw.gw_snr(gcat, net, gw.GW_DFLOAT)
    b, sb = gw.gw_snr(gcat, net, gw.GW_FP64)
    assert torch.equal(a, b) and torch.equal(sa, sb)
