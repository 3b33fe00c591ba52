"""FP64 Fisher pass with its Gram on the tensor cores (exact digit products)
against the same pass with every product on the FP64 pipe, and against the
oracle.

Both forms compute the Fisher matrix of Sec. 3.2 (Eqs. 3.1-3.3) in FP64; they
differ only in rounding: the tensor-core form is the exact Gram of the tangents
rounded to 56 bits relative to each column's maximum, summed exactly over the
digit pairs and rounded once to FP64, the FP64-pipe form rounds every one of its fused multiply-adds,
and the two evaluate the grid powers of v in different orders.  Elementwise
they agree to ~1e-14 of sqrt(Gamma_ii Gamma_jj); the bound below is 1e-12.

Cases cover one- and two-round work items (grids of 200 to 20000 points, items
of up to 128 points), both parameter counts (9: one L-shaped detector without
Earth rotation; 11: the triangle with rotation), a tabulated PSD, duty-factor
arm masks (empty interferometer slots), and a network wider than two
interferometers per point (which keeps the FP64-pipe kernel: the two settings
give identical results)."""
import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests import oracle_pool
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


@pytest.fixture(autouse=True)
def fp64_pipe_default():
    yield
    gw.gw_set_fp64_gram(False)


def _rel(F1, F2, np_):
    """max over events of |F1 - F2| / sqrt(F2_ii F2_jj), packed inputs [NPK, n]."""
    A = gw.unpack(F1, np_).cpu().numpy()
    B = gw.unpack(F2, np_).cpu().numpy()
    dg = np.sqrt(np.abs(np.einsum("eii->ei", B)))
    return float(np.max(np.abs(A - B) / (dg[:, :, None] * dg[:, None, :])))


def _both(gcat, net, np_, grad=False):
    up = torch.linspace(0.5, 1.5, gcat.n, dtype=torch.float64, device="cuda") if grad else None
    gw.gw_set_fp64_gram(True)
    a = gw.gw_fisher(gcat, net, np_, gw.GW_FP64, grad_snr=up)
    gw.gw_set_fp64_gram(False)
    b = gw.gw_fisher(gcat, net, np_, gw.GW_FP64, grad_snr=up)
    return a, b


CASES = {
    "c3_literal": ("c3", 60, "literal", None, 11),
    "c3_stress": ("c3", 12, "stress", None, 11),
    "c1_long": ("c1", 4, "literal", None, 11),
    "c0_L_norot": ("c0", 20, "literal", None, 9),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_gram_matches_fp64_pipe(name):
    cfg, n, grid, cap, np_ = CASES[name]
    cat, d, p = oracle_catalog(cfg, n, grid=grid, max_npts=cap)
    net = gw.Network(*gwcat.network(cfg))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    (F1, s1, st1, g1), (F2, s2, st2, g2) = _both(gcat, net, np_, grad=True)
    assert torch.equal(st1, st2) and int((st1 != 0).sum()) == 0
    r = _rel(F1, F2, np_)
    print(f"\n{name}: max |dGamma| / sqrt(Gii Gjj) = {r:.2e}, "
          f"SNR {torch.max(torch.abs(s1 / s2 - 1)).item():.2e}")
    assert r < 1e-12
    assert torch.max(torch.abs(s1 / s2 - 1)).item() < 1e-13
    # SNR gradient entries against their Cauchy-Schwarz scale grad_snr sqrt(Gamma_jj)
    # (phase parameters cancel to ~1e-15 of it)
    dgj = torch.sqrt(torch.stack([F2[j * np_ - j * (j - 1) // 2] for j in range(np_)]))
    up = torch.linspace(0.5, 1.5, gcat.n, dtype=torch.float64, device="cuda")
    assert torch.max(torch.abs(g1 - g2) / (dgj * up)).item() < 1e-12
    assert gw.gw_kernel_faults() == 0


def test_tensor_gram_against_oracle():
    """The tensor-core FP64 Fisher matrices and SNRs of a c3 catalog
    with one- and two-round items against the oracle's, at the FP64 parity
    bounds of the other tests (Gamma_ij 1e-8 of sqrt(Gamma_ii Gamma_jj), SNR
    1e-10: the oracle evaluates the same formulas in another order)."""
    cat, d, p = oracle_catalog("c3", 24, seed=20220714 + 41)
    det, psd, rot = gwcat.network("c3")
    F_or, s_or, _, st_or = oracle_pool.fisher(cat, det, psd, rot, 11)
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    gw.gw_set_fp64_gram(True)
    F, snr, st = gw.gw_fisher(gcat, gw.Network(det, psd, rot), 11, gw.GW_FP64)
    assert int((st != 0).sum()) == 0 and np.all(st_or == 0)
    A = gw.unpack(F, 11).cpu().numpy()
    dg = np.sqrt(np.einsum("eii->ei", F_or))
    rel = np.abs(A - F_or) / (dg[:, :, None] * dg[:, None, :])
    print(f"\nagainst the oracle: max |dGamma| / sqrt(Gii Gjj) = {rel.max():.2e}")
    assert rel.max() < 1e-8
    assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < 1e-10
    assert gw.gw_kernel_faults() == 0


def test_tensor_gram_tabulated_psd_and_arm_masks():
    cat, d, p = oracle_catalog("c3", 30, seed=20220714 + 42)
    masks = gwcat.draw_arm_masks(30, 3, 0.7, seed=9)
    det, rows, rot, tables = gwcat.network_tabulated("c3")
    for net, am in ((gw.Network(det, rows, rot, tables), None),
                    (gw.Network(*gwcat.network("c3")), masks)):
        gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, arm_mask=am)
        (F1, s1, st1), (F2, s2, st2) = _both(gcat, net, 11)
        assert torch.equal(st1, st2)
        ok = (st1 == 0).cpu().numpy()
        assert ok.sum() > 10
        # events with every arm off have zero Fisher matrices on both sides
        F1n, F2n = F1.cpu().numpy()[:, ok], F2.cpu().numpy()[:, ok]
        live = F2n[0] > 0
        assert _rel(torch.as_tensor(F1n[:, live]), torch.as_tensor(F2n[:, live]), 11) < 1e-12
        assert np.all(F1n[:, ~live] == 0)
    assert gw.gw_kernel_faults() == 0


def test_wider_network_keeps_fp64_pipe():
    """Four interferometers per point (triangle + two L): the setting does not
    apply and both calls run the FP64-pipe kernel (identical bits)."""
    cat, d, p = oracle_catalog("c4", 8, max_npts=600)
    net = gw.Network(*gwcat.network("c4"))
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    (F1, s1, st1), (F2, s2, st2) = _both(gcat, net, 11)
    assert torch.equal(F1, F2) and torch.equal(s1, s2)


def test_set_fp64_gram_rejects_bad_value():
    with pytest.raises(gw.GWError):
        gw._check(gw.load_library().gw_set_fp64_gram(gw.context(), 2), gw.context())
