"""Parity of the covariance tools (Sec. 4.1: CheckFisher, CovMatr and its
inversion options, the sky-localisation area; Sec. 4.2: fixParams, addPrior,
marginalisation) with the long-double CPU oracle, on the oracle's own Fisher
matrices of the seeded catalogs and on synthetic matrices with set spectra.

Both sides take the same FP64 input matrix; the GPU works in FP64, the oracle
in long double, so the tolerance on C_ij is (1e-12 + 1e-14 kappa) of
sqrt(C_ii C_jj), kappa the condition number of the normalised matrix.
"""
import numpy as np
import pytest
import torch

import gwcat
import oracle
from tests import oracle_pool
from tests.helpers import oracle_catalog, packed_index

pytestmark = pytest.mark.gpu

gw = pytest.importorskip("paper_2207_06910_gb300")


def pack(F):
    n, P, _ = F.shape
    return torch.as_tensor(np.stack([F[:, i, j] for i, j in packed_index(P)]), device="cuda")


def unpack_np(Cp, P):
    return gw.unpack(Cp, P).cpu().numpy()


def spectrum_matrices(P, n, lo, rng, scale=True):
    """Symmetric positive-definite matrices with eigenvalues log-spaced from 1 to
    10^-lo (factor >= 10 gaps) and random diagonal scales."""
    out = []
    for _ in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(P, P)))
        w = 10.0 ** -np.linspace(0, lo, P)
        D = np.diag(10.0 ** rng.uniform(-3, 3, P)) if scale else np.eye(P)
        out.append(D @ (Q * w) @ Q.T @ D)
    return np.stack(out)


@pytest.fixture(scope="module")
def fishers():
    """Oracle Fisher matrices of small seeded catalogs (kappa up to ~1e14)."""
    out = []
    for cfg, n, cap in (("c1", 4, 600), ("c2", 4, 600), ("c4", 3, None)):
        cat, _, _ = oracle_catalog(cfg, n, max_npts=cap)
        det, psd, rot = gwcat.network(cfg)
        F, s, err, st = oracle_pool.fisher(cat, det, psd, rot, 11)
        out.append(F)
    return np.concatenate(out)


def _cmp_status(st, so, kappa):
    """Status bits equal, except that FP64 Cholesky may find a matrix of
    condition number above 1e12 not positive definite where the long-double
    oracle does not (and then falls back to the SVD)."""
    soft = 1 | 128
    assert ((st & ~soft) == (so & ~soft)).all(), (st, so)
    firm = kappa < 1e12
    assert (st[firm] == so[firm]).all(), (st, so, kappa)


def _cmp_cov(Cg, Co, kappa, extra=0.0):
    for e in range(Cg.shape[0]):
        d = np.sqrt(np.abs(np.outer(np.diag(Co[e]), np.diag(Co[e]))))
        tol = 1e-12 + 1e-14 * kappa[e] + extra
        rel = np.max(np.abs(Cg[e] - Co[e]) / d)
        assert rel <= tol, (e, rel, kappa[e])


@pytest.mark.parametrize("method", [0, 1, 2, 5])
def test_covariance_methods_on_catalog_fishers(fishers, method):
    Fp = pack(fishers)
    C, cond, err, st = gw.gw_covariance(Fp, 11, method=method)
    Co, ko, eo, so = oracle.covariance(fishers, method=method)
    st = st.cpu().numpy()
    _cmp_status(st, so, ko)
    kg = cond.cpu().numpy()
    # the smallest eigenvalue carries an FP64 error of ~eps |A|: kappa to ~eps kappa
    assert np.all(np.abs(kg / ko - 1) <= 1e-6 + 2e-15 * ko), (kg, ko)
    ok = ((so | st) & 1) == 0
    _cmp_cov(unpack_np(C, 11)[ok], Co[ok], ko[ok])
    # inversion error of the same size as the oracle's (both ~kappa eps)
    e = err.cpu().numpy()[ok]
    assert np.all(e <= 1e-6 + 1e3 * eo[ok])


@pytest.mark.parametrize("method,thresh", [(3, 1e-4), (4, 1e-4), (2, 1e-4)])
def test_svd_floor_and_drop_on_set_spectra(method, thresh):
    """Spectra 1 .. 1e-6 (normalised matrices of unit diagonal: no rescaling),
    thresh 1e-4: the two smallest singular values are raised (3) or dropped (4)."""
    rng = np.random.default_rng(31)
    F = spectrum_matrices(11, 6, 6.0, rng, scale=False)
    # unit diagonal: normalise exactly on the host, symmetrically
    d = np.sqrt(np.einsum("eii->ei", F))
    F = F / (d[:, :, None] * d[:, None, :])
    F = 0.5 * (F + np.transpose(F, (0, 2, 1)))
    C, cond, err, st = gw.gw_covariance(pack(F), 11, method=method, thresh=thresh)
    Co, ko, eo, so = oracle.covariance(F, method=method, thresh=thresh)
    assert (st.cpu().numpy() == so).all()
    Cg = unpack_np(C, 11)
    for e in range(6):
        scale = np.max(np.abs(Co[e]))
        assert np.max(np.abs(Cg[e] - Co[e])) <= 1e-9 * scale


def test_fix_prior_submatrix_and_sky_area(fishers):
    keep = [0, 1, 2, 3, 4, 5, 6, 7, 8]            # fix the two last slots
    prior = np.zeros(11)
    prior[[3, 4, 5, 6, 8]] = 1.0 / (2 * np.pi ** 2)   # angles, as in the paper's example
    Fp = pack(fishers)
    C, cond, err, st = gw.gw_covariance(Fp, 11, keep=keep, prior=prior)
    Co, ko, eo, so = oracle.covariance(fishers, keep=keep, prior=prior)
    st = st.cpu().numpy()
    _cmp_status(st, so, ko)
    ok = ((so | st) & 1) == 0
    _cmp_cov(unpack_np(C, 9)[ok], Co[ok], ko[ok])
    # submatrix: bit-exact selection of packed entries
    sub = gw.gw_packed_submatrix(Fp, 11, [0, 2, 3, 4, 7])
    want = fishers[:, [0, 2, 3, 4, 7]][:, :, [0, 2, 3, 4, 7]]
    assert np.array_equal(unpack_np(sub, 5), want)
    # sky area from the GPU covariance, against the oracle's formula on the same C
    theta = torch.as_tensor(np.linspace(0.3, 2.8, fishers.shape[0]), device="cuda")
    Cfull, _, _, stf = gw.gw_covariance(Fp, 11)
    Cg = unpack_np(Cfull, 11)
    for units in ("SqDeg", "Sterad"):
        a = gw.gw_sky_area(Cfull, 11, theta, perc=90.0, units=units).cpu().numpy()
        ao = oracle.sky_area(Cg, 3, 4, theta.cpu().numpy(), perc=90.0, units=units)
        good = np.isfinite(ao)
        np.testing.assert_allclose(a[good], ao[good], rtol=1e-12)


def test_fisher_eig_values_vectors(fishers):
    rng = np.random.default_rng(32)
    F = np.concatenate([fishers, spectrum_matrices(11, 4, 8.0, rng)])
    for normalize in (True, False):
        w, V = gw.gw_fisher_eig(pack(F), 11, normalize=normalize)
        w = w.cpu().numpy().T
        V = V.cpu().numpy().T.reshape(-1, 11, 11)
        wo, Vo = oracle.fisher_eig(F, normalize=normalize)
        for e in range(F.shape[0]):
            d = np.sqrt(np.diag(F[e])) if normalize else np.ones(11)
            A = F[e] / np.outer(d, d)
            sc = np.max(np.abs(wo[e]))
            assert np.max(np.abs(w[e] - wo[e])) <= 1e-13 * sc
            # eigenvectors are unique where the eigenvalue is isolated: residual
            # and orthonormality always, agreement with the oracle where the gap
            # to the neighbours is large
            assert np.max(np.abs(A @ V[e] - V[e] * w[e])) <= 1e-12 * sc
            assert np.max(np.abs(V[e].T @ V[e] - np.eye(11))) <= 1e-12
            for k in range(11):
                gap = min([abs(wo[e, k] - wo[e, j]) for j in range(11) if j != k])
                if gap > 1e-3 * sc:
                    dv = min(np.max(np.abs(V[e][:, k] - Vo[e][:, k])),
                             np.max(np.abs(V[e][:, k] + Vo[e][:, k])))
                    assert dv <= 1e-10, (e, k, dv)


def test_not_pd_fallback_and_cond_max():
    rng = np.random.default_rng(33)
    Q, _ = np.linalg.qr(rng.normal(size=(9, 9)))
    Fi = ((Q * np.array([3, 2, 1.5, 1, 0.7, 0.5, -0.4, 0.3, 0.2])) @ Q.T)
    F = np.stack([Fi, Fi * 2.0])
    for method in (0, 1, 5):
        C, cond, err, st = gw.gw_covariance(pack(F), 9, method=method)
        Co, ko, eo, so = oracle.covariance(F, method=method)
        assert (st.cpu().numpy() == so).all(), (method, st, so)
        Cg = unpack_np(C, 9)
        if method == 0:
            assert np.isnan(Cg).all()
        else:
            np.testing.assert_allclose(Cg, Co, rtol=1e-10, atol=1e-12)
    G = spectrum_matrices(11, 2, 8.0, rng)
    C, cond, err, st = gw.gw_covariance(pack(G), 11, cond_max=1e5)
    assert (st.cpu().numpy() & 2).all() and torch.isnan(C).all()
    with pytest.raises(gw.GWError):
        gw.gw_covariance(pack(G), 11, method=9)
    with pytest.raises(gw.GWError):
        gw.gw_covariance(pack(G), 11, prior=[-1.0] * 11)


def test_perturb_fisher_bit_exact_and_stability(fishers):
    """perturb_Fisher (Sec. 4.1): elementwise products, compared exactly with the
    oracle's definition on the same random numbers; the covariance of the
    perturbed matrices moves by ~kappa eps, the stability check the paper runs."""
    rng = np.random.default_rng(34)
    F = 0.5 * (fishers + np.transpose(fishers, (0, 2, 1)))
    r = rng.uniform(-1, 1, F.shape)
    r = np.triu(r) + np.transpose(np.triu(r, 1), (0, 2, 1))
    Fp = gw.gw_perturb_fisher(pack(F), 11, pack(r), eps=1e-10)
    want = oracle.perturb_fisher(F, r, 1e-10)
    assert np.array_equal(unpack_np(Fp, 11), want)
    C0, k0, _, s0 = gw.gw_covariance(pack(F), 11)
    C1, _, _, s1 = gw.gw_covariance(Fp, 11)
    ok = ((s0 | s1).cpu().numpy() & 1) == 0
    d0 = np.sqrt(np.abs(np.einsum("eii->ei", unpack_np(C0, 11))))
    d1 = np.sqrt(np.abs(np.einsum("eii->ei", unpack_np(C1, 11))))
    rel = np.max(np.abs(d1 / d0 - 1), axis=1)
    assert np.all(rel[ok] <= 1e-10 * k0.cpu().numpy()[ok] + 1e-12)
