"""Shared test plumbing: seeded catalogs prepared by the oracle, and constants
retyped from their published values (used only by the pins)."""
import math

import numpy as np

import gwcat
import oracle

# published constants, retyped for the closed-form pins
TSUN = 4.925490947641267e-6          # G Msun / c^3 [s]
C_SI = 299792458.0
MPC_M = 3.085677581491367e22
R_EARTH = 6.371e6
T_SID = 86164.0905
OMEGA_E = 2 * math.pi / T_SID
GPC_S = 1e3 * MPC_M / C_SI


def oracle_catalog(cfg, n, grid="literal", seed=None, max_npts=None):
    """Seeded catalog for config ``cfg`` with parameters prepared by the oracle."""
    d = gwcat.draw(cfg, n, seed=seed, grid=grid)
    p = oracle.prepare(d["m1"], d["m2"], d["chi1"], d["chi2"], d["lam1"], d["lam2"],
                       d["dL_Mpc"], d["zflag"], d["tcoal"])
    ev = np.stack([p["Mc"], p["eta"], p["dL"], d["theta"], d["phi"], d["iota"], d["psi"],
                   p["tc"], d["Phic"], p["chi1z"], p["chi2z"], p["LamT"], p["dLamT"]], 1)
    rule = d["npts_rule"]
    if rule[0] == "efold":
        npts = oracle.grid_npts(d["fmin"], p["fisco"], *rule[1:])
    else:
        npts = d["npts"]
    if max_npts is not None:
        npts = np.minimum(npts, max_npts)
    return oracle.Catalog(ev, d["pset"], d["fmin"], p["fisco"], npts), d, p


def jks(lat, gam, zeta, theta, phi, psi, L):
    """Jaranowski-Krolak-Schutz closed-form pattern functions (bisector gamma from East)."""
    ds = math.pi / 2 - theta
    x = phi - L
    s2g, c2g = math.sin(2 * gam), math.cos(2 * gam)
    a = (s2g * (3 - math.cos(2 * lat)) * (3 - math.cos(2 * ds)) * math.cos(2 * x) / 16
         - c2g * math.sin(lat) * (3 - math.cos(2 * ds)) * math.sin(2 * x) / 4
         + s2g * math.sin(2 * lat) * math.sin(2 * ds) * math.cos(x) / 4
         - c2g * math.cos(lat) * math.sin(2 * ds) * math.sin(x) / 2
         + 3 * s2g * math.cos(lat) ** 2 * math.cos(ds) ** 2 / 4)
    b = (c2g * math.sin(lat) * math.sin(ds) * math.cos(2 * x)
         + s2g * (3 - math.cos(2 * lat)) * math.sin(ds) * math.sin(2 * x) / 4
         + c2g * math.cos(lat) * math.cos(ds) * math.cos(x)
         + s2g * math.sin(2 * lat) * math.cos(ds) * math.sin(x) / 2)
    fp = math.sin(zeta) * (a * math.cos(2 * psi) + b * math.sin(2 * psi))
    fx = math.sin(zeta) * (b * math.cos(2 * psi) - a * math.sin(2 * psi))
    return fp, fx


def amp0(Mc, dL):
    """f-independent factor of the leading-order amplitude, A = amp0 f^(-7/6)."""
    return math.sqrt(5 / 24) * math.pi ** (-2 / 3) * (Mc * TSUN) ** (5 / 6) / (dL * GPC_S)


def geom_grid(fmin, fmax, n):
    k = np.arange(n)
    f = fmin * (fmax / fmin) ** (k / (n - 1))
    w = np.zeros(n)
    w[1:] += 0.5 * np.diff(f)
    w[:-1] += 0.5 * np.diff(f)
    return f, w


def psd_eval(row, f):
    f0, scale, nt = row[0], row[1], int(row[2])
    return scale * sum(row[3 + j] * (f / f0) ** row[7 + j] for j in range(nt))


def packed_index(P):
    """(i, j) pairs of the packed upper triangle, row-major."""
    return [(i, j) for i in range(P) for j in range(i, P)]
