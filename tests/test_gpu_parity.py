"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every case uses the seeded synthetic catalogs of gwcat, prepared by the oracle,
and sizes that span several work items with a ragged tail.  Tolerances:
  FP64 path   SNR 1e-10 relative; Gamma_ij 1e-8 of sqrt(Gamma_ii Gamma_jj).
  mixed path  SNR 1e-5 relative; Gamma_ij 2e-6 of sqrt(Gamma_ii Gamma_jj)
              (tangents rounded to FP32 once per point: |dGamma_ij| <=
              2 u |g_i||g_j| with u = 6e-8, plus the FP32 Earth angle);
              sqrt(diag Gamma^-1) 1e-3 relative on events whose condition
              number is below 1e9, reported per decade above it.
"""
import math

import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests import oracle_pool
from tests.helpers import oracle_catalog

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")

CASES = {
    # name: (config, events, grid, npts cap)
    "c0": ("c0", 3, "literal", None),        # 2000 points, 1 L detector, no rotation
    "c1": ("c1", 4, "literal", 1100),        # 3 work items per event, ragged
    "c2": ("c2", 4, "literal", 1100),
    "c3": ("c3", 12, "literal", None),       # 200-277 points, BBH + BNS mixed
    "c3s": ("c3", 6, "stress", 1500),
    "c4": ("c4", 3, "literal", None),        # triangle + two L
}


def _setup(name):
    cfg, n, grid, cap = CASES[name]
    cat, d, p = oracle_catalog(cfg, n, grid=grid, max_npts=cap)
    det, psd, rot = gwcat.network(cfg)
    return cat, det, psd, rot, gwcat.N_PAR[cfg]


@pytest.fixture(scope="module")
def ref():
    """Oracle SNR / Fisher / inverse for every case, computed once in a pool."""
    out = {}
    for name in CASES:
        cat, det, psd, rot, P = _setup(name)
        F, s, err, st = oracle_pool.fisher(cat, det, psd, rot, P)
        s2, arm, st2 = oracle_pool.snr(cat, det, psd, rot)
        C, k, eps, sti = oracle.invert(F)
        out[name] = dict(cat=cat, det=det, psd=psd, rot=rot, P=P, F=F, snr=s, arm=arm, st=st,
                         C=C, kappa=k, inv_st=sti)
    return out


def _gpu_cat(cat):
    return gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts)


def _rel_fisher(Fg, F):
    dg = np.sqrt(np.einsum("eii->ei", F))
    return np.abs(Fg - F) / (dg[:, :, None] * dg[:, None, :])


def _arm_to_det(det, arm):
    """Oracle per-arm SNR -> per-detector SNR (triangle arms in quadrature)."""
    out, a = [], 0
    for r in det:
        k = 1 if int(r[4]) == 0 else 3
        out.append(np.sqrt(np.sum(arm[:, a:a + k] ** 2, axis=1)))
        a += k
    return np.array(out)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_snr(ref, name, prec):
    r = ref[name]
    cat = _gpu_cat(r["cat"])
    net = gw.Network(r["det"], r["psd"], r["rot"])
    snr, sdet, st = gw.gw_snr(cat, net, prec, per_detector=True)
    tol = 1e-10 if prec == 0 else 1e-5
    snr = snr.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    assert np.max(np.abs(snr / r["snr"] - 1)) < tol
    want = _arm_to_det(r["det"], r["arm"])
    assert np.max(np.abs(sdet.cpu().numpy() / want - 1)) < tol


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_fisher(ref, name, prec):
    r = ref[name]
    cat = _gpu_cat(r["cat"])
    net = gw.Network(r["det"], r["psd"], r["rot"])
    F, snr, st = gw.gw_fisher(cat, net, r["P"], prec)
    Fg = gw.unpack(F, r["P"]).cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    rel = _rel_fisher(Fg, r["F"])
    tol_f, tol_s = (1e-8, 1e-10) if prec == 0 else (2e-6, 1e-5)
    assert rel.max() < tol_f, f"max rel {rel.max():.3e} at {np.unravel_index(rel.argmax(), rel.shape)}"
    assert np.max(np.abs(snr.cpu().numpy() / r["snr"] - 1)) < tol_s


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c3s", "c4"])
@pytest.mark.parametrize("prec", [0, 1])
def test_covariance(ref, name, prec):
    """sqrt(diag C) of GPU Fisher + GPU inversion against the oracle's
    long-double inversion of its own Fisher."""
    r = ref[name]
    cat = _gpu_cat(r["cat"])
    net = gw.Network(r["det"], r["psd"], r["rot"])
    F, snr, st = gw.gw_fisher(cat, net, r["P"], prec)
    C, cond, err, sti = gw.gw_fisher_inverse(F, r["P"])
    Cg = gw.unpack(C, r["P"]).cpu().numpy()
    ok = (r["inv_st"] & (oracle.ST_NOT_PD | oracle.ST_NONFINITE)) == 0
    sg = np.sqrt(np.abs(np.einsum("eii->ei", Cg)))
    so = np.sqrt(np.abs(np.einsum("eii->ei", r["C"])))
    rel = np.max(np.abs(sg / so - 1), axis=1)
    kappa = r["kappa"]
    for e in np.nonzero(ok)[0]:
        if prec == 0:
            assert rel[e] < max(1e-9, 1e-12 * kappa[e]), (e, rel[e], kappa[e])
        elif kappa[e] < 1e9:
            assert rel[e] < 1e-3, (e, rel[e], kappa[e])
    fmt = {"float_kind": lambda x: f"{x:.2e}"}
    print(f"{name} prec={prec}: kappa {np.array2string(kappa, formatter=fmt)} "
          f"max rel sqrt(diag C) {np.array2string(rel, formatter=fmt)}")


@pytest.mark.parametrize("name", ["c0", "c1", "c2", "c4"])
def test_inversion_of_oracle_fisher(ref, name):
    """GPU inversion of the oracle's Fisher against the oracle's inversion of
    the same matrices (Sec. 4.1)."""
    r = ref[name]
    P = r["P"]
    F = r["F"]
    packed = np.stack([F[:, i, j] for i in range(P) for j in range(i, P)])
    Ft = torch.as_tensor(packed, device="cuda")
    C, cond, err, st = gw.gw_fisher_inverse(Ft, P)
    st = st.cpu().numpy()
    if name == "c0":
        # rank-deficient by construction: every event flagged
        assert np.all((st & (gw.ST_NOT_PD | gw.ST_ILL_COND)) != 0)
        return
    Cg = gw.unpack(C, P).cpu().numpy()
    for e in range(len(F)):
        k = r["kappa"][e]
        d = np.sqrt(np.abs(np.diag(r["C"][e])))
        rel = np.abs(Cg[e] - r["C"][e]) / np.outer(d, d)
        assert rel.max() < max(1e-12, 1e-14 * k), (e, rel.max(), k)
        # condition numbers: 1-norm (GPU) vs eigenvalue ratio (oracle) within P
        kg = cond.cpu().numpy()[e]
        assert k / P <= kg <= k * P * 1.0001
        assert (st[e] & gw.ST_ILL_COND != 0) == (kg > 1 / np.finfo(float).eps)


@pytest.mark.parametrize("name", ["c0", "c1", "c2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_snr_vjp(name, prec):
    cfg = CASES[name][0]
    cat, d, p = oracle_catalog(cfg, 3, max_npts=600)
    det, psd, rot = gwcat.network(cfg)
    P = gwcat.N_PAR[cfg]
    g_or = oracle_pool.snr_grad(cat, det, psd, rot, P)
    s_or, _ = oracle.snr(cat, det, psd, rot)
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    up = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    g = gw.gw_snr_vjp(gcat, net, P, up, prec).cpu().numpy().T
    want = g_or * up.cpu().numpy()[:, None]
    # natural scale of each parameter: SNR changes by O(SNR) over it
    scale = np.array([cat.ev[:, 0], np.full(3, 0.01), cat.ev[:, 2], np.ones(3), np.ones(3),
                      np.ones(3), np.ones(3), np.full(3, 1e3), np.ones(3)] +
                     ([np.ones(3), np.ones(3)] if P == 11 else [])).T
    rtol = 1e-7 if prec == 0 else 2e-5
    tol = rtol * (np.abs(want) + np.abs(up.cpu().numpy())[:, None] * s_or[:, None] / scale * 1e-3)
    assert np.all(np.abs(g - want) <= tol), np.max(np.abs(g - want) / tol)
    # the same VJP fused into the Fisher pass
    F, snr, st, gf = gw.gw_fisher(gcat, net, P, prec, grad_snr=up)
    gf = gf.cpu().numpy().T
    assert np.all(np.abs(gf - want) <= tol), np.max(np.abs(gf - want) / tol)


def test_snr_autograd_matches_vjp():
    cat, d, p = oracle_catalog("c1", 3, max_npts=300)
    det, psd, rot = gwcat.network("c1")
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    rows = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10]
    params = torch.tensor(cat.ev[:, rows].T.copy(), device="cuda", requires_grad=True)
    snr = gw.SNR.apply(params, gcat, net, 11, gw.GW_FP64)
    (snr * torch.tensor([1.0, 2.0, 3.0], device="cuda", dtype=torch.float64)).sum().backward()
    g = gw.gw_snr_vjp(gcat, net, 11, torch.tensor([1.0, 2.0, 3.0], device="cuda",
                                                  dtype=torch.float64))
    assert torch.allclose(params.grad, g, rtol=1e-14, atol=0)


def test_logdet_vjp_detangles():
    """d(sum_e log det Gamma_e)/d gamma of the two L detectors (five-interferometer
    network) against Richardson differences of the oracle's log det."""
    cat, d, p = oracle_catalog("c4", 2, max_npts=100)
    det, psd, rot = gwcat.network("c4")
    g_or, ld_or = oracle_pool.logdet_grad(cat, det, psd, rot, 11, [0, 1, 2])
    F_or, _, _, _ = oracle_pool.fisher(cat, det, psd, rot, 11)
    kappa = oracle.invert(F_or)[1].max()
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
    C, cond, err, sti = gw.gw_fisher_inverse(F, 11)
    g = gw.gw_logdet_vjp_detangles(gcat, net, 11, C, gw.GW_FP64).cpu().numpy()
    # tr(Gamma^-1 dGamma): an elementwise FP64 rounding u of the accumulated
    # Gamma moves it by ~u kappa; 2e-15 kappa covers sqrt(n) growth of u
    tol = 1e-6 + 2e-15 * kappa
    assert np.all(np.abs(g - g_or) < tol * (np.abs(g_or) + 1.0)), (g, g_or, kappa)
    # a closed triangle is invariant under rotation in its plane: d/d gamma_T = 0
    assert abs(g_or[0]) < 1e-12 and abs(g[0]) < tol


def test_logdet_vjp_detangles_masked():
    """The log-det gradient for a subset of the detectors (the two L detectors
    of the five-interferometer network, which is what the orientation study
    asks for) equals the full call's entries bit for bit, since a detector's
    gradient sums only its own interferometers; the other entries are NaN.  An
    empty catalog gives 0 for the selected detectors; a mask selecting no
    detector of the network is rejected."""
    cat, d, p = oracle_catalog("c4", 40, max_npts=300)
    det, psd, rot = gwcat.network("c4")
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_MIXED)
    C, cond, err, sti = gw.gw_fisher_inverse(F, 11)
    full = gw.gw_logdet_vjp_detangles(gcat, net, 11, C).cpu().numpy()
    assert np.all(np.isfinite(full))
    for mask in (0b110, 0b010, 0b001, 0b111, 0b1101):
        g = gw.gw_logdet_vjp_detangles(gcat, net, 11, C, det_mask=mask).cpu().numpy()
        for k in range(3):
            if (mask >> k) & 1:
                assert g[k] == full[k], (mask, k)
            else:
                assert np.isnan(g[k]), (mask, k)
    with pytest.raises(gw.GWError):
        gw.gw_logdet_vjp_detangles(gcat, net, 11, C, det_mask=0b1000)
    empty = gcat.select(torch.empty(0, dtype=torch.int64, device="cuda"))
    g0 = gw.gw_logdet_vjp_detangles(empty, net, 11, C, det_mask=0b110).cpu().numpy()
    assert np.isnan(g0[0]) and g0[1] == 0.0 and g0[2] == 0.0


# ---------------------------------------------------------------- edges
def test_grid_edges_against_oracle():
    """Grid lengths around the work-item size (32 lanes x 16 points)."""
    cat0, d, p = oracle_catalog("c0", 1)
    lens = [2, 3, 31, 32, 33, 511, 512, 513, 1024, 1025]
    ev = np.repeat(cat0.ev[:1], len(lens), axis=0)
    ev[:, 9:] = 0
    cat = oracle.Catalog(ev, 0, 10.0, cat0.fmax[0], np.array(lens, dtype=np.int32))
    det, psd, rot = gwcat.network("c0")
    F_or, s_or, _, _ = oracle_pool.fisher(cat, det, psd, rot, 9)
    gcat = _gpu_cat(cat)
    net = gw.Network(det, psd, rot)
    for prec, tf, ts in ((0, 1e-8, 1e-10), (1, 2e-6, 1e-5)):
        F, snr, st = gw.gw_fisher(gcat, net, 9, prec)
        assert np.all(st.cpu().numpy() == 0)
        assert np.max(np.abs(snr.cpu().numpy() / s_or - 1)) < ts
        assert _rel_fisher(gw.unpack(F, 9).cpu().numpy(), F_or).max() < tf


def test_bad_events_flagged_and_isolated():
    cat, d, p = oracle_catalog("c1", 6, max_npts=200)
    ev = cat.ev.copy()
    fmin, fmax, npts = cat.fmin.copy(), cat.fmax.copy(), cat.npts.copy()
    pset = cat.pset.copy()
    ev[0, 1] = 0.26            # eta > 1/4
    ev[1, 2] = -1.0            # dL <= 0
    fmax[2] = 1.0              # fmax < fmin
    npts[3] = 1                # one point
    ev[4, 3] = np.nan          # non-finite angle
    det, psd, rot = gwcat.network("c1")
    net = gw.Network(det, psd, rot)
    gcat = gw.Catalog.from_numpy(ev, pset, fmin, fmax, npts)
    F, snr, st = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
    st = st.cpu().numpy()
    assert st[0] & gw.ST_BAD_PARAM and st[1] & gw.ST_BAD_PARAM and st[4] & gw.ST_BAD_PARAM
    assert st[2] & gw.ST_EMPTY_GRID and st[3] & gw.ST_EMPTY_GRID and st[5] == 0
    Fh = F.cpu().numpy()
    assert np.all(np.isnan(Fh[:, :5])) and np.all(np.isfinite(Fh[:, 5]))
    good = oracle.Catalog(ev[5:], pset[5:], fmin[5:], fmax[5:], npts[5:])
    F_or, s_or, _, _ = oracle.fisher(good, det, psd, rot, 11)
    assert _rel_fisher(gw.unpack(F, 11).cpu().numpy()[5:], F_or).max() < 1e-8
    # a 9-parameter request on 11-parameter events is a per-event error
    F9, s9, st9 = gw.gw_fisher(gw.Catalog.from_numpy(ev[5:], pset[5:], fmin[5:], fmax[5:],
                                                     npts[5:]), net, 9)
    assert st9.cpu().numpy()[0] & gw.ST_BAD_PARAM


def test_empty_catalog_and_argument_errors():
    det, psd, rot = gwcat.network("c1")
    net = gw.Network(det, psd, rot)
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    t = {k: z for k in gw.Catalog.FIELDS}
    cat = gw.Catalog(t, torch.empty(0, dtype=torch.int8, device="cuda"), z, z,
                     torch.empty(0, dtype=torch.int32, device="cuda"))
    F, snr, st = gw.gw_fisher(cat, net, 11)
    assert F.numel() == 0
    with pytest.raises(gw.GWError):
        gw.gw_fisher(cat, net, 10)
    bad = gw.Network(np.array([[0.1, 0.2, 0.3, 1.5, 7, 0]]), psd, rot)
    with pytest.raises(gw.GWError):
        gw.gw_fisher(cat, bad, 11)


# ---------------------------------------------------------------- full size
def test_prepare_matches_oracle_full_c3():
    d = gwcat.draw("c3")
    cat = gw.gw_prepare_catalog(d, d["npts_rule"])
    p = oracle.prepare(d["m1"], d["m2"], d["chi1"], d["chi2"], d["lam1"], d["lam2"],
                       d["dL_Mpc"], d["zflag"], d["tcoal"])
    for k in ("Mc", "eta", "dL", "chi1z", "chi2z", "LamT", "dLamT", "tc"):
        got = cat.t[k].cpu().numpy()
        # FP64 against long double over a few operations: a few ulp
        assert np.allclose(got, p[k], rtol=4e-15, atol=4e-15 * np.max(np.abs(p[k]))), k
    assert np.allclose(cat.fmax.cpu().numpy(), p["fisco"], rtol=1e-13, atol=0)
    # grid length: ceil(40 ln(f_ISCO / f_min)) from the oracle's own f_ISCO.  An
    # argument within a few ulp of an integer may round to either side in the
    # GPU's double precision; those events are excused and counted.
    per, lo, hi = d["npts_rule"][1:]
    npts_or = oracle.grid_npts(d["fmin"], p["fisco"], per, lo, hi)
    x = per * np.log(p["fisco"] / d["fmin"])
    near = np.abs(x - np.rint(x)) <= 16 * np.finfo(float).eps * np.abs(x)
    near &= (np.rint(x) >= lo) & (np.rint(x) <= hi + 1)
    got = cat.npts.cpu().numpy()
    bad = (got != npts_or) & ~near
    print(f"grid lengths: {near.sum()} of {len(x)} arguments within 16 ulp of an integer")
    assert not bad.any(), np.nonzero(bad)[0][:10]
    assert np.all(np.abs(got - npts_or)[near] <= 1)


@pytest.mark.parametrize("grid", ["literal", "stress"])
def test_full_size_c3_sampled_and_invariants(grid):
    """The 1e5-event catalog in the launch configuration of the benchmark:
    invariants on every event, oracle parity on sampled events."""
    d = gwcat.draw("c3", grid=grid)
    cat = gw.gw_prepare_catalog(d, d["npts_rule"])
    det, psd, rot = gwcat.network("c3")
    net = gw.Network(det, psd, rot)
    rng = np.random.default_rng(5)
    npts = cat.npts.cpu().numpy()
    pick = rng.choice(np.nonzero(npts <= 1500)[0], 3, replace=False)
    ev = np.stack([cat.t[k].cpu().numpy() for k in gw.Catalog.FIELDS], 1)
    sub = oracle.Catalog(ev[pick], d["pset"][pick], d["fmin"][pick],
                         cat.fmax.cpu().numpy()[pick], npts[pick])
    F_or, s_or, _, _ = oracle_pool.fisher(sub, det, psd, rot, 11)
    for prec, tf in ((0, 1e-8), (1, 2e-6)):
        F, snr, st = gw.gw_fisher(cat, net, 11, prec)
        assert int((st != 0).sum()) == 0
        s2 = snr ** 2
        k_pp = 8 * 11 - 8 * 7 // 2 + 0     # packed index of (8, 8)
        k_dd = 2 * 11 - 2 * 1 // 2 + 0     # packed index of (2, 2)
        itol = 1e-12 if prec == 0 else 1e-6
        assert torch.max(torch.abs(F[k_pp] / s2 - 1)).item() < itol
        dl = cat.t["dL"]
        assert torch.max(torch.abs(F[k_dd] * dl * dl / s2 - 1)).item() < itol
        Fs = gw.unpack(F[:, torch.as_tensor(pick, device="cuda")], 11).cpu().numpy()
        assert _rel_fisher(Fs, F_or).max() < tf


def test_reserve_async_graph_and_overflow():
    """gw_reserve: the asynchronous path replayed from a CUDA graph gives the
    synchronous results; events past the reserved work items are flagged."""
    cat, d, p = oracle_catalog("c3", 300)
    det, psd, rot = gwcat.network("c3")
    net = gw.Network(det, psd, rot)
    gcat = _gpu_cat(cat)
    up = torch.ones(gcat.n, dtype=torch.float64, device="cuda")
    F0, s0, st0, g0 = gw.gw_fisher(gcat, net, 11, gw.GW_MIXED, grad_snr=up)
    items = gw.work_items(gcat.npts)
    try:
        gw.gw_reserve(gcat.n, items, 1)
        gw.gw_fisher(gcat, net, 11, gw.GW_MIXED, grad_snr=up)      # warm outside capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            F1, s1, st1, g1 = gw.gw_fisher(gcat, net, 11, gw.GW_MIXED, grad_snr=up)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(F1, F0) and torch.equal(s1, s0) and torch.equal(g1, g0)
        assert torch.equal(st1, st0)
        # too few items reserved: trailing events overflow, the rest are unchanged
        gw.gw_reserve(gcat.n, items - 7, 1)
        F2, s2, st2 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
        F3, s3, st3 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
        st2 = st2.cpu().numpy()
        over = (st2 & gw.ST_OVERFLOW) != 0
        assert 1 <= over.sum() <= 7 and over[-1] and not over[0]
        assert np.all(np.isnan(F2.cpu().numpy()[:, over]))
        gw.gw_reserve(0, 0, 0)
        F4, s4, st4 = gw.gw_fisher(gcat, net, 11, gw.GW_FP64)
        assert torch.equal(F2[:, ~torch.as_tensor(over, device="cuda")],
                           F4[:, ~torch.as_tensor(over, device="cuda")])
    finally:
        gw.gw_reserve(0, 0, 0)


@pytest.mark.parametrize("masked", [False, True])
def test_snr_vjp_detector_angles(masked):
    """d(sum_e w_e SNR_e)/d gamma_d (gw_snr_vjp's detector-orientation output) on
    the five-interferometer network against Richardson central differences of the
    oracle's SNR over each detector's orientation; with a duty-factor mask that
    switches one triangle arm off for one event the triangle's entry is no longer
    zero (a closed triangle's SNR does not change when it turns in its plane)."""
    cat, d, p = oracle_catalog("c4", 3, max_npts=300)
    det, psd, rot = gwcat.network("c4")
    mask = None
    if masked:
        mask = np.array([0b11110, 0b11111, 0b11111], dtype=np.uint32)   # arm 0 off, event 0
        cat = oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, mask)
    w = np.array([1.0, -2.0, 0.5])

    def snr_at(k, gam):
        dd = det.copy()
        dd[k, 2] = gam
        return oracle.snr(cat, dd, psd, rot)[0]

    want = []
    for k in range(len(det)):
        g0, h = det[k, 2], 2e-3
        dh = lambda hh: (snr_at(k, g0 + hh) - snr_at(k, g0 - hh)) / (2 * hh)
        want.append(np.sum(w * (4 * dh(h / 2) - dh(h)) / 3))
    want = np.array(want)
    gcat = gw.Catalog.from_numpy(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, arm_mask=mask)
    net = gw.Network(det, psd, rot)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    s0 = oracle.snr(cat, det, psd, rot)[0]
    scale = np.sum(np.abs(w) * s0)              # d SNR / d gamma is O(SNR) per radian
    for prec, tol in ((gw.GW_FP64, 1e-8), (gw.GW_MIXED, 2e-5)):
        g, gg = gw.gw_snr_vjp(gcat, net, 11, wt, prec, det_gamma=True)
        gg = gg.cpu().numpy()
        assert np.all(np.abs(gg - want) <= tol * scale), (prec, gg, want)
        if not masked:
            assert abs(gg[0]) <= tol * scale and abs(want[0]) <= 1e-8 * scale
        else:
            assert abs(want[0]) > 1e-4 * scale
