"""Parity of the duty factor (per-event arm masks), row selection and the SNR
detection gate with the CPU oracle, through the C ABI.

Duty factor: Sec. 3.2 and the duty_factor option of Sec. 5 (each detector and
each arm of a triangle on or off for a whole event).  Gate: the snr_th option
of Sec. 5.  Tolerances are those of test_gpu_parity.py; events with every arm
off must give exactly zero SNR and Fisher on both sides.
"""
import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests import oracle_pool
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")

# c4 network: triangle (arms 0, 1, 2), L (arm 3), L (arm 4)
MASKS = np.array([0b11111, 0, 0b00001, 0b00110, 0b01011, 0b10111, 0b11000, 0b00111,
                  0b11110, 0b01101], dtype=np.uint32)


def _gpu_cat(cat):
    return gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts,
                                 arm_mask=cat.arm_mask)


@pytest.fixture(scope="module")
def masked():
    cat, d, p = oracle_catalog("c4", len(MASKS), seed=20220714 + 900)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, MASKS)
    det, psd, rot = gwcat.network("c4")
    F, s, err, st = oracle_pool.fisher(cat, det, psd, rot, 11)
    s2, arm, st2 = oracle_pool.snr(cat, det, psd, rot)
    return dict(cat=cat, det=det, psd=psd, rot=rot, F=F, snr=s, arm=arm)


def _arm_to_det(det, arm):
    out, a = [], 0
    for r in det:
        k = 1 if int(r[4]) == 0 else 3
        out.append(np.sqrt(np.sum(arm[:, a:a + k] ** 2, axis=1)))
        a += k
    return np.array(out)


@pytest.mark.parametrize("prec", [0, 1])
def test_duty_masks_snr_and_fisher(masked, prec):
    r = masked
    gcat = _gpu_cat(r["cat"])
    net = gw.Network(r["det"], r["psd"], r["rot"])
    tol_f, tol_s = (1e-8, 1e-10) if prec == 0 else (2e-6, 1e-5)
    snr, sdet, st = gw.gw_snr(gcat, net, prec, per_detector=True)
    snr, sdet = snr.cpu().numpy(), sdet.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    on = r["snr"] > 0
    assert snr[~on].tolist() == [0.0] * int((~on).sum())
    assert np.max(np.abs(snr[on] / r["snr"][on] - 1)) < tol_s
    want = _arm_to_det(r["det"], r["arm"])
    assert np.all(np.abs(sdet - want) <= tol_s * r["snr"][None, :])
    F, snr_f, st = gw.gw_fisher(gcat, net, 11, prec)
    Fg = gw.unpack(F, 11).cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for e in range(len(MASKS)):
        if not on[e]:
            assert np.all(Fg[e] == 0.0) and snr_f[e].item() == 0.0
            continue
        dg = np.sqrt(np.diag(r["F"][e]))
        rel = np.abs(Fg[e] - r["F"][e]) / np.outer(dg, dg)
        assert rel.max() < tol_f, (e, bin(MASKS[e]), rel.max())


@pytest.mark.parametrize("prec", [0, 1])
def test_duty_masks_snr_vjp(prec):
    cat, d, p = oracle_catalog("c4", 4, seed=20220714 + 901, max_npts=300)
    masks = np.array([0b00001, 0b11000, 0, 0b10110], dtype=np.uint32)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)
    det, psd, rot = gwcat.network("c4")
    g_or = oracle_pool.snr_grad(cat, det, psd, rot, 11)
    s_or, _ = oracle.snr(cat, det, psd, rot)
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    up = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")
    upn = up.cpu().numpy()
    want = g_or * upn[:, None]
    scale = np.array([cat.ev[:, 0], np.full(4, 0.01), cat.ev[:, 2]] + [np.ones(4)] * 4 +
                     [np.full(4, 1e3)] + [np.ones(4)] * 3).T
    rtol = 1e-7 if prec == 0 else 2e-5
    tol = rtol * (np.abs(want) + np.abs(upn)[:, None] * s_or[:, None] / scale * 1e-3)
    g = gw.gw_snr_vjp(gcat, net, 11, up, prec).cpu().numpy().T
    assert np.all(g[2] == 0.0)                     # no arm on: SNR identically zero
    assert np.all(np.abs(g - want) <= tol), np.max(np.abs(g - want) / np.maximum(tol, 1e-300))
    F, snr, st, gf = gw.gw_fisher(gcat, net, 11, prec, grad_snr=up)
    gf = gf.cpu().numpy().T
    assert np.all(gf[2] == 0.0)
    assert np.all(np.abs(gf - want) <= tol), np.max(np.abs(gf - want) / np.maximum(tol, 1e-300))


def test_duty_masks_logdet_vjp():
    """With the second L off for every event its orientation gradient is exactly
    zero; the triangle with one arm off is no longer rotation invariant."""
    cat, d, p = oracle_catalog("c4", 2, seed=20220714 + 902, max_npts=100)
    masks = np.array([0b01110, 0b01101], dtype=np.uint32)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)
    det, psd, rot = gwcat.network("c4")
    g_or, ld_or = oracle_pool.logdet_grad(cat, det, psd, rot, 11, [0, 1, 2])
    F_or, _, _, _ = oracle_pool.fisher(cat, det, psd, rot, 11)
    kappa = oracle.invert(F_or)[1].max()
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
    C, cond, err, sti = gw.gw_fisher_inverse(F, 11)
    g = gw.gw_logdet_vjp_detangles(gcat, net, 11, C, gw.GW_FP64).cpu().numpy()
    tol = 1e-6 + 2e-15 * kappa
    assert g[2] == 0.0 and g_or[2] == 0.0
    assert np.all(np.abs(g - g_or) < tol * (np.abs(g_or) + 1.0)), (g, g_or, kappa)
    assert abs(g_or[0]) > 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_row_selection_equals_gathered_catalog(prec):
    """A catalog view through sel gives bit-identical results to a catalog whose
    columns were gathered on the host (same rows, same arithmetic)."""
    cat, d, p = oracle_catalog("c3", 40, seed=20220714 + 903)
    masks = gwcat.draw_arm_masks(40, 3, 0.8, seed=5)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)
    det, psd, rot = gwcat.network("c3")
    net = gw.Network(det, psd, rot)
    idx = np.array([37, 2, 2, 0, 19, 11, 39, 5], dtype=np.int64)
    full = _gpu_cat(cat)
    view = full.select(torch.as_tensor(idx, device="cuda"))
    gath = _gpu_cat(cat.subset(idx))
    assert view.n == len(idx)
    up = torch.linspace(-1, 1, len(idx), dtype=torch.float64, device="cuda")
    a = gw.gw_fisher(view, net, 11, prec, grad_snr=up)
    b = gw.gw_fisher(gath, net, 11, prec, grad_snr=up)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    sa = gw.gw_snr(view, net, prec)
    sb = gw.gw_snr(gath, net, prec)
    assert torch.equal(sa[0], sb[0])


def test_select_snr_is_the_oracle_rule_bit_exact():
    """The gate's decisions are integer results: compared exactly with the
    oracle's rule applied to the same SNR array (NaN, ties, empty results)."""
    rng = np.random.default_rng(11)
    s = rng.uniform(0, 40, 5000)
    s[::97] = np.nan
    s[10] = 12.0
    s[11] = np.nextafter(12.0, 13.0)
    t = torch.as_tensor(s, device="cuda")
    for th in (12.0, -1.0, 50.0, 0.0):
        sel = gw.gw_select_snr(t, th).cpu().numpy()
        assert sel.tolist() == oracle.select_snr(s, th).tolist()
    assert gw.gw_select_snr(t[:0], 1.0).numel() == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_gated_pipeline_against_oracle(prec):
    """SNR pass over a catalog with duty-factor masks, gate at SNR > 12, Fisher
    of the selected events only; the selected set and their Fisher matrices
    against the oracle's (the gate applied to the GPU SNR on both sides)."""
    cat, d, p = oracle_catalog("c3", 30, seed=20220714 + 904)
    masks = gwcat.draw_arm_masks(30, 3, 0.7, seed=6)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)
    det, psd, rot = gwcat.network("c3")
    net = gw.Network(det, psd, rot)
    gcat = _gpu_cat(cat)
    snr, st = gw.gw_snr(gcat, net, prec)
    sel = gw.gw_select_snr(snr, 12.0)
    sel_np = sel.cpu().numpy()
    assert sel_np.tolist() == oracle.select_snr(snr.cpu().numpy(), 12.0).tolist()
    assert 0 < len(sel_np) < 30
    F, s_sel, st = gw.gw_fisher(gcat.select(sel), net, 11, prec)
    sub = cat.subset(sel_np)
    F_or, s_or, _, _ = oracle_pool.fisher(sub, det, psd, rot, 11)
    tol_f, tol_s = (1e-8, 1e-10) if prec == 0 else (2e-6, 1e-5)
    assert np.max(np.abs(s_sel.cpu().numpy() / s_or - 1)) < tol_s
    Fg = gw.unpack(F, 11).cpu().numpy()
    dg = np.sqrt(np.einsum("eii->ei", F_or))
    rel = np.abs(Fg - F_or) / (dg[:, :, None] * dg[:, None, :])
    assert rel.max() < tol_f


@pytest.mark.parametrize("prec", [0, 1])
def test_largest_network_with_masks(prec):
    """Eight detectors (three triangles and five L-shaped ones: 14 arms, 20
    interferometer entries of the 24 the library holds) with random arm masks,
    against the oracle; a network beyond the capacity is refused."""
    D = np.pi / 180
    det = np.array([[40.5 * D, 9.4 * D, 0.0, 60 * D, 1, 0],
                    [50.7 * D, 5.9 * D, 10 * D, 60 * D, 1, 0],
                    [-30 * D, 120 * D, 35 * D, 60 * D, 1, 1],
                    [46.5 * D, -119.4 * D, 171 * D, 90 * D, 0, 1],
                    [30.6 * D, -90.8 * D, 242.7 * D, 90 * D, 0, 1],
                    [43.6 * D, 10.5 * D, 115.6 * D, 90 * D, 0, 1],
                    [36.4 * D, 137.3 * D, 15.4 * D, 90 * D, 0, 0],
                    [19.6 * D, 77.0 * D, 287.4 * D, 90 * D, 0, 0]])
    _, psd, rot = gwcat.network("c4")
    cat, d, p = oracle_catalog("c3", 3, seed=20220714 + 905, max_npts=150)
    masks = gwcat.draw_arm_masks(3, 14, 0.7, seed=7)
    cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)
    F_or, s_or, _, _ = oracle_pool.fisher(cat, det, psd, rot, 11)
    net = gw.Network(det, psd, rot)
    F, snr, st = gw.gw_fisher(_gpu_cat(cat), net, 11, prec)
    tol_f, tol_s = (1e-8, 1e-10) if prec == 0 else (2e-6, 1e-5)
    assert np.all(st.cpu().numpy() == 0)
    assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < tol_s
    Fg = gw.unpack(F, 11).cpu().numpy()
    dg = np.sqrt(np.einsum("eii->ei", F_or))
    assert (np.abs(Fg - F_or) / (dg[:, :, None] * dg[:, None, :])).max() < tol_f
    big = np.concatenate([det[:3], det[:2], det[3:6]])      # five triangles: 28 entries
    with pytest.raises(gw.GWError):
        gw.gw_fisher(_gpu_cat(cat), gw.Network(big, psd, rot), 11, prec)
