"""Tabulated noise curves (Sec. 3.1: a detector's PSD or ASD read from a table,
the psd_path / is_ASD options) through the C ABI against the oracle's
log-log interpolation of the same tables.

The tables sample the configurations' analytic PSD shape on 2000 log-spaced
frequencies (gwcat.network_tabulated); the five-interferometer network reads
its two curves as an amplitude spectral density.  Tolerances as for the analytic
PSD: FP64 SNR 1e-10 relative and Gamma_ij 1e-8 of sqrt(Gamma_ii Gamma_jj);
mixed 1e-5 and 2e-6.  A table that covers part of the band leaves the points
outside it with zero weight; a table that breaks its rules gives NaN."""
import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests import oracle_pool
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")

CASES = {"c3": ("c3", 10, None, False), "c4_asd": ("c4", 4, 300, True),
         "c1": ("c1", 3, 700, False)}


def _rel_fisher(Fg, F):
    dg = np.sqrt(np.einsum("eii->ei", F))
    return np.abs(Fg - F) / (dg[:, :, None] * dg[:, None, :])


@pytest.mark.parametrize("name", list(CASES))
def test_tabulated_psd_against_oracle(name):
    cfg, n, cap, asd = CASES[name]
    cat, d, p = oracle_catalog(cfg, n, max_npts=cap)
    det, rows, rot, tables = gwcat.network_tabulated(cfg, asd=asd)
    F_or, s_or, _, st_or = oracle_pool.fisher(cat, det, rows, rot, 11, tables)
    assert np.all(st_or == 0)
    # the tabulated curve differs from the analytic one only by interpolation
    det0, psd0, _ = gwcat.network(cfg)
    F_an, s_an, _, _ = oracle_pool.fisher(cat, det0, psd0, rot, 11)
    assert np.max(np.abs(s_or / s_an - 1)) < 1e-4
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    net = gw.Network(det, rows, rot, tables)
    for prec, tf, ts in ((gw.GW_FP64, 1e-8, 1e-10), (gw.GW_MIXED, 2e-6, 1e-5)):
        F, snr, st = gw.gw_fisher(gcat, net, 11, prec)
        assert int((st != 0).sum()) == 0
        assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < ts
        assert _rel_fisher(gw.unpack(F, 11).cpu().numpy(), F_or).max() < tf
        s2, st2 = gw.gw_snr(gcat, net, prec)
        assert np.max(np.abs(s2.cpu().numpy() / s_or - 1)) < ts


def test_partial_table_is_blind_outside():
    """A table covering 2.5..60 Hz: grid points outside have zero weight."""
    cat, d, p = oracle_catalog("c3", 6)
    det, psd, rot = gwcat.network("c3")
    f = np.geomspace(2.5, 60.0, 300)
    shape = (f / 10.0) ** -4.0 + 2.0 + 2.0 * (f / 10.0) ** 2
    tables = [(f, shape, False)]
    rows = [[1.0, 1e-49, -1, 0, 0, 0, 0, 0, 0, 0, 0]]
    s_or, _, _ = oracle_pool.snr(cat, det, rows, rot, tables)
    F_or, _, _, _ = oracle_pool.fisher(cat, det, rows, rot, 11, tables)
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    net = gw.Network(det, rows, rot, tables)
    assert np.all(s_or > 0) and np.all(cat.fmax > 2.5)
    for prec, tf, ts in ((gw.GW_FP64, 1e-8, 1e-10), (gw.GW_MIXED, 2e-6, 1e-5)):
        F, snr, st = gw.gw_fisher(gcat, net, 11, prec)
        assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < ts
        assert _rel_fisher(gw.unpack(F, 11).cpu().numpy(), F_or).max() < tf
    # the full-band SNR is larger: the points outside the table are left out
    s_full, _ = oracle.snr(cat, det, psd, rot)
    assert np.all(s_full > s_or)


def test_bad_table_gives_nan():
    cat, d, p = oracle_catalog("c3", 3)
    det, psd, rot = gwcat.network("c3")
    f = np.geomspace(1.0, 1e4, 50)
    f[20] = f[19]                       # not strictly increasing
    net = gw.Network(det, [[1.0, 1e-49, -1, 0, 0, 0, 0, 0, 0, 0, 0]], rot,
                     [(f, np.ones(50), False)])
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)
    for prec in (gw.GW_FP64, gw.GW_MIXED):
        snr, st = gw.gw_snr(gcat, net, prec)
        assert torch.all(torch.isnan(snr))
    with pytest.raises(gw.GWError):
        bad = gw.Network(det, [[1.0, 1e-49, -1, 0, 0, 0, 0, 0, 0, 0, 0]], rot,
                         [(f[:1], np.ones(1), False)])
        gw.gw_snr(gcat, bad, gw.GW_FP64)
