"""Seeded synthetic catalogs and detector networks for the Fisher-forecast path.

This module draws random numbers and holds configuration data only (detector
sites, PSD coefficients, grid rules).  It contains none of the method's
arithmetic: masses are not combined, redshift is not applied, no waveform or
grid quantity is computed here.  Both the CPU oracle (``oracle/``) and the CUDA
library consume its output, and it imports neither.

Populations follow the five synthetic workloads that stand in for the
population catalogs of the paper's companion study (not available here):

* ``c0``  100 BNS, one L-shaped interferometer, no Earth rotation, 2000 points
          from 10 Hz, 9 Fisher parameters.
* ``c1``  1e4 BBH (source-frame masses, redshifted with a linear Hubble law),
          triangle, rotation on, 5000 points from 2 Hz, 11 parameters (spins).
* ``c2``  1e4 tidal BNS, triangle, rotation on, 1e4 points from 2 Hz,
          11 parameters (Lambda-tilde, delta-Lambda-tilde).
* ``c3``  1e5 events, 70 % c1-BBH / 30 % c2-BNS, per-event grid from 2 Hz to
          f_ISCO; point count either by the 40-points-per-e-fold rule clamped to
          [200, 20000] ("literal") or log-uniform on [200, 20000] ("stress").
* ``c4``  1e6 events drawn as c3 on five interferometers (triangle + two L).
"""
from __future__ import annotations

import math

import numpy as np

DEG = math.pi / 180.0
SEED_BASE = 20220714

# PSD row: f0, scale, nterm, c0..c3, p0..p3   ->  S(f) = scale * sum c_j (f/f0)^p_j
PSD_3TERM = [10.0, 1e-49, 3, 1.0, 2.0, 2.0, 0.0, -4.0, 0.0, 2.0, 0.0]
PSD_3TERM_HALF = [10.0, 0.5e-49, 3, 1.0, 2.0, 2.0, 0.0, -4.0, 0.0, 2.0, 0.0]

# detector row: lat, lon, gamma, zeta [rad], shape (0 L, 1 triangle), psd index
DET_L_C0 = [43.0 * DEG, 10.0 * DEG, 20.0 * DEG, 90.0 * DEG, 0, 0]
DET_TRI = [40.5 * DEG, 9.4 * DEG, 0.0, 60.0 * DEG, 1, 0]
DET_L_A = [46.0 * DEG, -119.0 * DEG, 126.0 * DEG, 90.0 * DEG, 0, 1]
DET_L_B = [30.0 * DEG, -90.0 * DEG, 198.0 * DEG, 90.0 * DEG, 0, 1]

NETWORKS = {
    "c0": dict(det=np.array([DET_L_C0]), psd=np.array([PSD_3TERM]), rotation=0),
    "c1": dict(det=np.array([DET_TRI]), psd=np.array([PSD_3TERM]), rotation=1),
    "c2": dict(det=np.array([DET_TRI]), psd=np.array([PSD_3TERM]), rotation=1),
    "c3": dict(det=np.array([DET_TRI]), psd=np.array([PSD_3TERM]), rotation=1),
    "c4": dict(det=np.array([DET_TRI, DET_L_A, DET_L_B]),
               psd=np.array([PSD_3TERM, PSD_3TERM_HALF]), rotation=1),
}

SIZES = {"c0": 100, "c1": 10_000, "c2": 10_000, "c3": 100_000, "c4": 1_000_000}

# grid rule: fmin and either a fixed point count or ("efold", per_efold, lo, hi)
GRIDS = {
    "c0": dict(fmin=10.0, rule=("fixed", 2000)),
    "c1": dict(fmin=2.0, rule=("fixed", 5000)),
    "c2": dict(fmin=2.0, rule=("fixed", 10000)),
    "c3": dict(fmin=2.0, rule=("efold", 40.0, 200, 20000)),
    "c4": dict(fmin=2.0, rule=("efold", 40.0, 200, 20000)),
}

N_PAR = {"c0": 9, "c1": 11, "c2": 11, "c3": 11, "c4": 11}


def _angles(rng, n):
    return dict(
        theta=np.arccos(rng.uniform(-1.0, 1.0, n)),
        phi=rng.uniform(0.0, 2 * math.pi, n),
        iota=np.arccos(rng.uniform(-1.0, 1.0, n)),
        psi=rng.uniform(0.0, math.pi, n),
        tcoal=rng.uniform(0.0, 1.0, n),
        Phic=rng.uniform(0.0, 2 * math.pi, n),
    )


def _bns(rng, n, tidal):
    d = dict(
        m1=rng.uniform(1.1, 2.0, n), m2=rng.uniform(1.1, 2.0, n),
        chi1=rng.uniform(-0.05, 0.05, n), chi2=rng.uniform(-0.05, 0.05, n),
        lam1=rng.uniform(0.0, 1000.0, n) if tidal else np.zeros(n),
        lam2=rng.uniform(0.0, 1000.0, n) if tidal else np.zeros(n),
        dL_Mpc=rng.uniform(50.0, 500.0, n),
        zflag=np.zeros(n, dtype=np.uint8),
        pset=np.full(n, 2 if tidal else 0, dtype=np.int8),
    )
    d.update(_angles(rng, n))
    return d


def _bbh(rng, n):
    a, b = 100.0, 20000.0
    u = rng.uniform(0.0, 1.0, n)
    d = dict(
        m1=rng.uniform(5.0, 80.0, n), m2=rng.uniform(5.0, 80.0, n),
        chi1=rng.uniform(-0.8, 0.8, n), chi2=rng.uniform(-0.8, 0.8, n),
        lam1=np.zeros(n), lam2=np.zeros(n),
        # p(dL) ~ dL^2 on [a, b] by inverse CDF
        dL_Mpc=np.cbrt(a ** 3 + u * (b ** 3 - a ** 3)),
        zflag=np.ones(n, dtype=np.uint8),
        pset=np.full(n, 1, dtype=np.int8),
    )
    d.update(_angles(rng, n))
    return d


def draw(config: str, n: int | None = None, seed: int | None = None, grid: str = "literal"):
    """Raw seeded draws for ``config`` (c0..c4).  Returns a dict of numpy arrays
    (masses in Msun, dL in Mpc, tcoal in sidereal days, angles in rad, pset,
    zflag) plus the grid description ``fmin`` and ``npts_rule`` / ``npts``."""
    if config not in SIZES:
        raise ValueError(f"unknown config {config!r}")
    n = SIZES[config] if n is None else int(n)
    idx = int(config[1])
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + idx if seed is None else seed))
    if config == "c0":
        d = _bns(rng, n, tidal=False)
    elif config == "c1":
        d = _bbh(rng, n)
    elif config == "c2":
        d = _bns(rng, n, tidal=True)
    else:
        is_bbh = rng.uniform(0.0, 1.0, n) < 0.7
        nb = int(is_bbh.sum())
        a = _bbh(rng, nb)
        b = _bns(rng, n - nb, tidal=True)
        d = {}
        for k in a:
            out = np.empty(n, dtype=a[k].dtype)
            out[is_bbh] = a[k]
            out[~is_bbh] = b[k]
            d[k] = out
    g = GRIDS[config]
    d["fmin"] = np.full(n, g["fmin"])
    rule = g["rule"]
    if config in ("c3", "c4") and grid == "stress":
        # the 100x spread of per-event grid lengths, independent of the physics
        lo, hi = 200.0, 20000.0
        d["npts"] = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(np.int32)
        d["npts_rule"] = ("given",)
    elif rule[0] == "fixed":
        d["npts"] = np.full(n, rule[1], dtype=np.int32)
        d["npts_rule"] = rule
    else:
        d["npts"] = None
        d["npts_rule"] = rule
    d["config"] = config
    d["n_par"] = N_PAR[config]
    return d


def network(config: str):
    """Detector table [n_det, 6], PSD table [n_psd, 11], Earth-rotation flag."""
    net = NETWORKS[config]
    return net["det"].copy(), net["psd"].copy(), net["rotation"]


def network_tabulated(config: str, n_table: int = 2000, asd: bool = False,
                      f_lo: float = 1.0, f_hi: float = 1e4):
    """The network of ``config`` with every PSD given as a table (the psd_path
    option of the paper's detectors): the configuration's power-sum shape
    sum_j c_j (f/f0)^p_j sampled on ``n_table`` log-spaced frequencies in
    [f_lo, f_hi], as PSD values or (``asd``) their square roots; the row keeps
    its scale.  Returns (det, psd rows with nterm = -(k+1) for table k,
    rotation, tables = [(f, values, asd), ...])."""
    det, psd, rot = network(config)
    f = np.geomspace(f_lo, f_hi, n_table)
    rows, tables = [], []
    for k, r in enumerate(psd):
        shape = sum(r[3 + j] * (f / r[0]) ** r[7 + j] for j in range(int(r[2])))
        tables.append((f.copy(), np.sqrt(shape) if asd else shape, asd))
        rows.append([1.0, r[1], -(k + 1), 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    return det, np.array(rows), rot, tables


def draw_arm_masks(n: int, n_arms: int, duty: float, seed: int | None = None) -> np.ndarray:
    """Duty-factor draws (one Bernoulli trial per event and arm): bit a of the
    returned uint32 mask of event e is set, i.e. arm a of the expanded network
    (an L-shaped detector is one arm, a triangle three consecutive ones) is on
    for the whole event, with probability ``duty``, independently."""
    if not 0 < n_arms <= 32:
        raise ValueError("1..32 arms")
    rng = np.random.default_rng(SEED_BASE + 500 if seed is None else seed)
    on = rng.random((n, n_arms)) < duty
    return (on.astype(np.uint64) << np.arange(n_arms, dtype=np.uint64)).sum(1).astype(np.uint32)

