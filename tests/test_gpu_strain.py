"""Parity of the materialised strain h_a(f_k) = Q_a exp(i Phi_a) (Sec. 2.2
waveform projected as in Sec. 3.1, Earth rotation and Doppler phase) with the
oracle's long-double strain, arm by arm, on seeded events.

Tolerances: the phase reaches 1e6 rad, so FP64 rounding of Psi and of the grid
frequencies moves it by ~1e-9 rad: |dh| <= 1e-8 max|h| (FP64 sine/cosine) and
<= 3e-7 max|h| (FP32 sine/cosine of the FP64-reduced phase).
"""
import ctypes

import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def _gpu_cat(cat):
    return gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts,
                                 arm_mask=cat.arm_mask)


@pytest.mark.parametrize("cfg,n,cap,masks", [
    ("c0", 3, 700, None),                      # L detector, no rotation
    ("c1", 3, 900, None),                      # triangle, rotation, 2 Hz
    ("c2", 2, 900, None),                      # tidal BNS: phase up to ~1e6 rad
    ("c4", 4, None, [0b11111, 0b00110, 0b11000, 0]),
])
@pytest.mark.parametrize("prec", [0, 1])
def test_strain_against_oracle(cfg, n, cap, masks, prec):
    cat, _, _ = oracle_catalog(cfg, n, max_npts=cap)
    if masks is not None:
        cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts,
                             np.array(masks, dtype=np.uint32))
    det, psd, rot = gwcat.network(cfg)
    net = gw.Network(det, psd, rot)
    re, im, freq, off, st = gw.gw_strain(_gpu_cat(cat), net, prec)
    h = (re + 1j * im).cpu().numpy()
    off = off.cpu().numpy()
    freq = freq.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    assert off.tolist() == [0] + np.cumsum(cat.npts).tolist()
    tol = 1e-8 if prec == 0 else 3e-7
    for e in range(n):
        f_or, h_or = oracle.strain(cat.ev[e], cat.fmin[e], cat.fmax[e], int(cat.npts[e]), det, rot)
        seg = slice(off[e], off[e + 1])
        np.testing.assert_allclose(freq[seg], f_or, rtol=1e-14)
        scale = np.max(np.abs(h_or))
        for a in range(h_or.shape[0]):
            on = masks is None or (masks[e] >> a) & 1
            if not on:
                assert np.all(h[a, seg] == 0)
                continue
            err = np.max(np.abs(h[a, seg] - h_or[a]))
            assert err <= tol * scale, (e, a, err / scale)


def test_strain_triangle_arms_sum_to_zero_and_checks():
    """The three arms of a closed triangle sum to zero (the geometric identity the
    paper uses for the triangle, Sec. 3.3); a wrong total_points is rejected."""
    cat, _, _ = oracle_catalog("c1", 2, max_npts=400)
    det, psd, rot = gwcat.network("c1")
    net = gw.Network(det, psd, rot)
    gcat = _gpu_cat(cat)
    re, im, freq, off, st = gw.gw_strain(gcat, net, 0)
    h = (re + 1j * im).cpu().numpy()
    assert np.max(np.abs(h.sum(axis=0))) <= 1e-13 * np.max(np.abs(h))
    lib = gw.load_library()
    c = gcat.struct()
    total = int(cat.npts.sum())
    st = lib.gw_strain(gw.context(), ctypes.byref(c), ctypes.byref(net.net), 0, total + 1,
                       gw._ptr(re), gw._ptr(im), None, None, None, gw._stream())
    assert st == 1 and b"total_points" in lib.gw_last_error(gw.context())


def test_strain_of_selected_rows_equals_gathered_catalog():
    """gw_strain through a row selection gives the bit-identical output of a
    catalog gathered on the host (same rows, same arithmetic)."""
    cat, _, _ = oracle_catalog("c1", 5, max_npts=300)
    det, psd, rot = gwcat.network("c1")
    net = gw.Network(det, psd, rot)
    idx = np.array([4, 0, 2], dtype=np.int64)
    view = _gpu_cat(cat).select(torch.as_tensor(idx, device="cuda"))
    gath = _gpu_cat(cat.subset(idx))
    for prec in (0, 1):
        a = gw.gw_strain(view, net, prec)
        b = gw.gw_strain(gath, net, prec)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
