"""CPU oracle for the Fisher-forecast hot path of GWFAST (arXiv:2207.06910).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py``; never by the library.
The arithmetic lives in ``gw_oracle.c`` (plain C, long double, derivatives by
Richardson-extrapolated central differences); this module only marshals numpy
arrays through ctypes.  See the header of ``gw_oracle.c`` for which section or
equation of the paper each function follows.

Event rows are 13 doubles in the order of ``PARAMS``:
``Mc [Msun], eta, dL [Gpc], theta, phi, iota, psi [rad], tc [s], Phic [rad],
chi1z, chi2z, LambdaTilde, deltaLambdaTilde``.
A detector row is ``lat, lon, gamma, zeta [rad], shape (0 = L, 1 = triangle),
psd index``; a PSD row is ``f0, scale, nterm, c0..c3, p0..p3`` with
``S_n(f) = scale * sum_j c_j (f/f0)^p_j``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

PARAMS = ("Mc", "eta", "dL", "theta", "phi", "iota", "psi", "tc", "Phic",
          "chi1z", "chi2z", "LamT", "dLamT")

ST_NOT_PD, ST_COND_GT_MAX, ST_NONFINITE, ST_EMPTY_GRID, ST_BAD_PARAM, ST_ILL_COND = 1, 2, 4, 8, 16, 32
ST_SVD_FALLBACK = 128

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gw_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgworacle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math) into ``oracle/_build``."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_prepare.argtypes = [i64] + [P] * 9 + [P] * 9
        lib.or_set_fd_target.argtypes = [d]
        lib.or_grid_npts.argtypes = [i64, P, P, d, i32, i32, P]
        lib.or_psi_pn.argtypes = [d] * 7
        lib.or_psi_pn.restype = d
        lib.or_tau_star.argtypes = [d] * 3
        lib.or_tau_star.restype = d
        lib.or_antenna.argtypes = [d] * 7 + [P, P]
        lib.or_strain.argtypes = [P, d, d, i32, i32, P, i32, P, P, P]
        lib.or_snr.argtypes = [i64, P, P, P, P, P, i32, P, i32, P, i32, P, P, P]
        lib.or_fisher.argtypes = [i64, P, P, P, P, P, P, i32, P, i32, P, i32, i32, P, P, P, P]
        lib.or_invert.argtypes = [i64, i32, P, d, P, P, P, P]
        lib.or_snr_grad.argtypes = [i64, P, P, P, P, P, P, i32, P, i32, P, i32, i32, P]
        lib.or_logdet_grad_gamma.argtypes = [i64, P, P, P, P, P, P, i32, P, i32, P, i32, i32, i32,
                                             P, d, P, P]
        lib.or_fisher_eig.argtypes = [i64, i32, P, i32, P, P]
        lib.or_covariance.argtypes = [i64, i32, P, ctypes.c_uint32, P, i32, d, d, P, P, P, P]
        lib.or_sky_area.argtypes = [i64, i32, P, i32, i32, P, d, i32, P]
        lib.or_set_psd_tables.argtypes = [i32, P, P, P, P]
        lib.or_psd_eval.argtypes = [P, i32, d]
        lib.or_psd_eval.restype = d
        if lib.or_abi_version() != 4:
            raise RuntimeError("stale oracle build: rebuild with oracle.build(force=True)")
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def n_arms(det) -> int:
    det = np.asarray(det, dtype=np.float64).reshape(-1, 6)
    return int(sum(1 if int(r[4]) == 0 else 3 for r in det))


def prepare(m1, m2, chi1, chi2, lam1, lam2, dL_Mpc, zflag, tcoal):
    """Raw draws -> Fisher parameters (Sec. 2.1, Eq. 2.2; f_ISCO of Sec. 2.2)."""
    lib = _load()
    n = len(m1)
    ins = [_f64(m1), _f64(m2), _f64(chi1), _f64(chi2),
           None if lam1 is None else _f64(lam1), None if lam2 is None else _f64(lam2),
           _f64(dL_Mpc), np.ascontiguousarray(zflag, dtype=np.uint8), _f64(tcoal)]
    outs = [np.empty(n) for _ in range(9)]
    lib.or_prepare(n, *[_p(a) for a in ins], *[_p(a) for a in outs])
    keys = ("Mc", "eta", "dL", "chi1z", "chi2z", "LamT", "dLamT", "tc", "fisco")
    return dict(zip(keys, outs))


def set_psd_tables(tables) -> None:
    """Tabulated noise curves (Sec. 3.1, the psd_path / is_ASD options):
    ``tables`` is a list of (f, values, is_asd); a PSD row ``table_row(k, scale)``
    then reads table k with log-log linear interpolation, zero weight outside
    the tabulated range."""
    n = np.array([len(t[0]) for t in tables], dtype=np.int64)
    f = _f64(np.concatenate([t[0] for t in tables])) if tables else np.zeros(1)
    v = _f64(np.concatenate([t[1] for t in tables])) if tables else np.zeros(1)
    asd = np.array([1 if t[2] else 0 for t in tables], dtype=np.int32)
    if _load().or_set_psd_tables(len(tables), _p(n), _p(f), _p(v), _p(asd)) != 0:
        raise ValueError("tables need >= 2 points, f > 0 strictly increasing, values > 0")


def psd_eval(psd, idx: int, f: float) -> float:
    """S_n(f) of row ``idx`` of a PSD table (rows as in ``snr``)."""
    psd = _f64(psd).reshape(-1, 11)
    return _load().or_psd_eval(_p(psd), int(idx), float(f))


def table_row(k: int, scale: float = 1.0):
    """PSD row reading table k (see set_psd_tables), times ``scale``."""
    return [1.0, float(scale), -(k + 1), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]


def set_fd_target(target: float = 0.1) -> None:
    """Phase excursion (rad) of the first Richardson step; 0.1 by default."""
    _load().or_set_fd_target(float(target))


def grid_npts(fmin, fmax, per_efold, lo, hi):
    """Per-event grid length by the points-per-e-fold rule, clamped to [lo, hi]."""
    fmin, fmax = _f64(fmin), _f64(fmax)
    out = np.empty(len(fmin), dtype=np.int32)
    _load().or_grid_npts(len(fmin), _p(fmin), _p(fmax), float(per_efold), int(lo), int(hi), _p(out))
    return out


def psi_pn(Mc, eta, chi1, chi2, LT, dLT, f):
    return _load().or_psi_pn(Mc, eta, chi1, chi2, LT, dLT, f)


def tau_star(Mc, eta, f):
    return _load().or_tau_star(Mc, eta, f)


def antenna(lat, L, gamma, zeta, theta, phi, psi):
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().or_antenna(lat, L, gamma, zeta, theta, phi, psi, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def strain(ev, fmin, fmax, npts, det, rotation):
    """Complex strain of every arm: returns (f [npts], h [n_arms, npts])."""
    det = _f64(det).reshape(-1, 6)
    na = n_arms(det)
    f = np.empty(npts)
    re = np.empty((na, npts))
    im = np.empty((na, npts))
    _load().or_strain(_p(_f64(ev)), fmin, fmax, npts, det.shape[0], _p(det), int(rotation),
                      _p(f), _p(re), _p(im))
    return f, re + 1j * im


class Catalog:
    """Event rows [n,13], parameter set [n], grid (fmin, fmax, npts) per event, and
    optional duty-factor arm masks [n] (bit a = arm a of the expanded network is
    on; None = every arm on)."""

    def __init__(self, ev, pset, fmin, fmax, npts, arm_mask=None):
        self.ev = _f64(ev).reshape(-1, 13)
        n = self.ev.shape[0]
        self.pset = np.ascontiguousarray(np.broadcast_to(pset, (n,)), dtype=np.int8)
        self.fmin = _f64(np.broadcast_to(fmin, (n,)))
        self.fmax = _f64(np.broadcast_to(fmax, (n,)))
        self.npts = np.ascontiguousarray(np.broadcast_to(npts, (n,)), dtype=np.int32)
        self.arm_mask = (None if arm_mask is None else
                         np.ascontiguousarray(np.broadcast_to(arm_mask, (n,)), dtype=np.uint32))

    def __len__(self):
        return self.ev.shape[0]

    def subset(self, idx):
        return Catalog(self.ev[idx], self.pset[idx], self.fmin[idx], self.fmax[idx], self.npts[idx],
                       None if self.arm_mask is None else self.arm_mask[idx])


def snr(cat: Catalog, det, psd, rotation, per_arm=False):
    det = _f64(det).reshape(-1, 6)
    psd = _f64(psd).reshape(-1, 11)
    n = len(cat)
    na = n_arms(det)
    out = np.empty(n)
    arm = np.empty((n, na)) if per_arm else None
    st = np.empty(n, dtype=np.int32)
    _load().or_snr(n, _p(cat.ev), _p(cat.fmin), _p(cat.fmax), _p(cat.npts), _p(cat.arm_mask),
                   det.shape[0],
                   _p(det), psd.shape[0], _p(psd), int(rotation), _p(out), _p(arm), _p(st))
    return (out, arm, st) if per_arm else (out, st)


def fisher(cat: Catalog, det, psd, rotation, n_par):
    """Full Fisher matrices [n, P, P], SNR [n], Richardson error bar [n], status [n]."""
    det = _f64(det).reshape(-1, 6)
    psd = _f64(psd).reshape(-1, 11)
    n = len(cat)
    F = np.empty((n, n_par, n_par))
    s = np.empty(n)
    err = np.empty(n)
    st = np.empty(n, dtype=np.int32)
    _load().or_fisher(n, _p(cat.ev), _p(cat.pset), _p(cat.fmin), _p(cat.fmax), _p(cat.npts),
                      _p(cat.arm_mask), det.shape[0], _p(det), psd.shape[0], _p(psd), int(rotation), n_par,
                      _p(F), _p(s), _p(err), _p(st))
    return F, s, err, st


def invert(F, cond_max=1e50):
    """Covariance [n,P,P], condition number (eigenvalues of the normalised matrix),
    inversion error max|Gamma C - 1|, status bits."""
    F = _f64(F)
    n, P, _ = F.shape
    C = np.empty_like(F)
    k = np.empty(n)
    e = np.empty(n)
    st = np.empty(n, dtype=np.int32)
    _load().or_invert(n, P, _p(F), float(cond_max), _p(C), _p(k), _p(e), _p(st))
    return C, k, e, st


def snr_grad(cat: Catalog, det, psd, rotation, n_par):
    det = _f64(det).reshape(-1, 6)
    psd = _f64(psd).reshape(-1, 11)
    n = len(cat)
    g = np.empty((n, n_par))
    _load().or_snr_grad(n, _p(cat.ev), _p(cat.pset), _p(cat.fmin), _p(cat.fmax), _p(cat.npts),
                        _p(cat.arm_mask), det.shape[0], _p(det), psd.shape[0], _p(psd), int(rotation), n_par, _p(g))
    return g


def logdet_grad_gamma(cat: Catalog, det, psd, rotation, n_par, dets, step0=0.05):
    """d(sum_e log det Gamma_e)/d gamma_d for detector indices ``dets``; also the
    per-event log det at the fiducial orientation."""
    det = _f64(det).reshape(-1, 6)
    psd = _f64(psd).reshape(-1, 11)
    dets = np.ascontiguousarray(dets, dtype=np.int32)
    n = len(cat)
    g = np.empty(len(dets))
    ld = np.empty(n)
    _load().or_logdet_grad_gamma(n, _p(cat.ev), _p(cat.pset), _p(cat.fmin), _p(cat.fmax),
                                 _p(cat.npts), _p(cat.arm_mask), det.shape[0], _p(det), psd.shape[0], _p(psd),
                                 int(rotation), n_par, len(dets), _p(dets), float(step0),
                                 _p(g), _p(ld))
    return g, ld


def select_snr(snr, threshold):
    """Detection gate (Sec. 5, the snr_th option): the indices, in increasing
    order, of the events whose network SNR exceeds the threshold; Fisher
    matrices are computed for these events only.  NaN SNRs are never selected."""
    snr = np.asarray(snr, dtype=np.float64)
    return np.flatnonzero(snr > threshold).astype(np.int64)


# inversion methods of covariance() (the invMethodIn options of Sec. 4.1)
INV_CHO, INV_CHO_SVD, INV_SVD, INV_SVD_TRUNC, INV_SVD_REG, INV_LU = range(6)


def fisher_eig(F, normalize=True):
    """Eigenvalues [n, P] (ascending) and eigenvectors [n, P, P] (columns) of each
    Fisher matrix, normalised by sqrt(diag) if ``normalize`` (CheckFisher)."""
    F = _f64(F)
    n, P, _ = F.shape
    w = np.empty((n, P))
    V = np.empty((n, P, P))
    _load().or_fisher_eig(n, P, _p(F), int(normalize), _p(w), _p(V))
    return w, V


def covariance(F, keep=None, prior=None, method=INV_CHO_SVD, thresh=1e-15, cond_max=1e50):
    """CovMatr with fixParams (``keep``: indices of the parameters kept) and
    addPrior (``prior``: [P] values added to the diagonal of kept parameters).
    Returns cov [n, Pk, Pk], condition number, inversion error, status."""
    F = _f64(F)
    n, P, _ = F.shape
    keep = list(range(P)) if keep is None else sorted(keep)
    mask = 0
    for i in keep:
        mask |= 1 << int(i)
    Pk = len(keep)
    C = np.empty((n, Pk, Pk))
    k = np.empty(n)
    e = np.empty(n)
    st = np.empty(n, dtype=np.int32)
    pr = None if prior is None else _f64(prior)
    _load().or_covariance(n, P, _p(F), mask, _p(pr), int(method), float(thresh), float(cond_max),
                          _p(C), _p(k), _p(e), _p(st))
    return C, k, e, st


def sky_area(C, i_theta, i_phi, theta, perc=90.0, units="SqDeg"):
    """Delta Omega_perc% of each event (Sec. 4.1), 'SqDeg' or 'Sterad'."""
    C = _f64(C)
    n, P, _ = C.shape
    out = np.empty(n)
    _load().or_sky_area(n, P, _p(C), int(i_theta), int(i_phi), _p(_f64(theta)), float(perc),
                        1 if units == "SqDeg" else 0, _p(out))
    return out


def perturb_fisher(F, r, eps=1e-10):
    """perturb_Fisher (Sec. 4.1): every element of each Fisher matrix perturbed at
    the eps-th relative decimal, Gamma'_ij = Gamma_ij (1 + eps r_ij), with r the
    caller's random numbers in [-1, 1] taken from the upper triangle (r_ji = r_ij,
    so Gamma' stays symmetric).  F [n, P, P], r [n, P, P]."""
    F = _f64(F)
    r = _f64(r)
    iu = np.triu_indices(F.shape[1])
    rs = np.zeros_like(r)
    rs[:, iu[0], iu[1]] = r[:, iu[0], iu[1]]
    rs = rs + np.transpose(rs, (0, 2, 1)) - rs * np.eye(F.shape[1])
    return F * (1.0 + eps * rs)

