"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: a published
identity between two independent coefficient tables, a closed form, a second
published form of the same quantity, a symmetry, or a library routine on a
special case.  A dropped term, wrong sign or transposed index in the oracle
fails at least one of them.  No GPU is needed.
"""
import math

import numpy as np
import pytest

import gwcat
import oracle
from tests.helpers import (OMEGA_E, R_EARTH, C_SI, amp0, geom_grid, jks, oracle_catalog,
                           psd_eval)

RNG = np.random.default_rng(7)


def richardson(fun, x, h, levels=4):
    """Richardson-extrapolated central difference of a scalar function (test-side)."""
    R = []
    for m in range(levels):
        d = h / 2 ** m
        R.append([(fun(x + d) - fun(x - d)) / (2 * d)])
    for j in range(1, levels):
        for m in range(j, levels):
            R[m].append(R[m][j - 1] + (R[m][j - 1] - R[m - 1][j - 1]) / (4 ** j - 1))
    return R[-1][-1]


# ---------------------------------------------------------------- waveform tables
@pytest.mark.parametrize("Mc,eta", [(1.2, 0.2499), (1.5, 0.23), (30.0, 0.2), (8.0, 0.1)])
def test_phase_and_tau_tables_agree(Mc, eta):
    """dPsi/df = -2 pi tau*(f) for the non-spinning 3.5PN tables (stationary phase:
    the time-frequency relation of Buonanno et al. 2009, cited in Sec. 2.2)."""
    fisco = 1 / (6 ** 1.5 * math.pi * Mc * eta ** -0.6 * 4.925490947641267e-6)
    for f in np.geomspace(3.0, 0.8 * fisco, 6):
        dpsi = richardson(lambda x: oracle.psi_pn(Mc, eta, 0, 0, 0, 0, x), f, 1e-3 * f)
        tau = oracle.tau_star(Mc, eta, f)
        assert abs(dpsi + 2 * math.pi * tau) <= 1e-9 * abs(2 * math.pi * tau)


def test_chirp_mass_scaling():
    """At fixed eta, Psi depends on Mc f only and tau* = Mc x function(Mc f)."""
    for _ in range(5):
        Mc, eta, lam = RNG.uniform(1, 40), RNG.uniform(0.1, 0.25), RNG.uniform(0.5, 2)
        f = 5.0
        a = oracle.psi_pn(lam * Mc, eta, 0.3, -0.2, 0, 0, f)
        b = oracle.psi_pn(Mc, eta, 0.3, -0.2, 0, 0, lam * f)
        assert abs(a - b) <= 1e-13 * abs(a)
        ta, tb = oracle.tau_star(lam * Mc, eta, f), lam * oracle.tau_star(Mc, eta, lam * f)
        assert abs(ta - tb) <= 1e-13 * abs(ta)


def _v(Mc, eta, f):
    return (math.pi * Mc * 4.925490947641267e-6 * eta ** -0.6 * f) ** (1 / 3)


def test_spin_terms_match_chis_chia_form():
    """The spin-orbit coefficient written per body equals the (chi_s, chi_a) form
    (Eq. (2.1) of the paper defines chi_s, chi_a), with spin-spin 79/8 eta chi1 chi2."""
    for _ in range(6):
        Mc, eta = RNG.uniform(2, 30), RNG.uniform(0.1, 0.249)
        c1, c2 = RNG.uniform(-0.9, 0.9, 2)
        f = RNG.uniform(3, 20)
        d = math.sqrt(1 - 4 * eta)
        cs, ca = (c1 + c2) / 2, (c1 - c2) / 2
        beta = 113 / 12 * (cs + d * ca - 76 / 113 * eta * cs)
        sigma = 79 / 8 * eta * c1 * c2
        v = _v(Mc, eta, f)
        expect = 3 / (128 * eta * v ** 5) * (4 * beta * v ** 3 - 10 * sigma * v ** 4)
        got = oracle.psi_pn(Mc, eta, c1, c2, 0, 0, f) - oracle.psi_pn(Mc, eta, 0, 0, 0, 0, f)
        assert abs(got - expect) <= 1e-7 * abs(expect) + 1e-9


def test_tidal_phase_matches_per_body_form():
    """Lambda-tilde / delta-Lambda-tilde from Eq. (2.2) inserted in the 5PN+6PN
    tidal phase equal the per-body tidal phase (Flanagan-Hinderer 5PN,
    Vines-Flanagan-Hinderer 6PN)."""
    n = 8
    m1, m2 = RNG.uniform(1.0, 2.2, n), RNG.uniform(1.0, 2.2, n)
    L1, L2 = RNG.uniform(0, 2000, n), RNG.uniform(0, 2000, n)
    z = np.zeros(n)
    p = oracle.prepare(m1, m2, z, z, L1, L2, np.full(n, 100.0), np.zeros(n, np.uint8), z)
    for e in range(n):
        a, b, la, lb = m1[e], m2[e], L1[e], L2[e]
        if b > a:
            a, b, la, lb = b, a, lb, la
        M = a + b
        X = (a / M, b / M)
        Lam = (la, lb)
        eta = p["eta"][e]
        f = RNG.uniform(20, 300)
        v = _v(p["Mc"][e], eta, f)
        s5 = sum(24 * (1 + 11 * X[1 - i]) * X[i] ** 4 * Lam[i] for i in range(2))
        s6 = sum((15895 / 28 - 4595 / 28 * X[i] - 5715 / 14 * X[i] ** 2 + 325 / 7 * X[i] ** 3)
                 * X[i] ** 4 * Lam[i] for i in range(2))
        expect = 3 / (128 * eta) * (-s5 * v ** 5 - s6 * v ** 7)
        got = (oracle.psi_pn(p["Mc"][e], eta, 0, 0, p["LamT"][e], p["dLamT"][e], f)
               - oracle.psi_pn(p["Mc"][e], eta, 0, 0, 0, 0, f))
        assert abs(got - expect) <= 1e-8 * abs(expect)


def test_lambda_tilde_special_cases():
    """Eq. (2.2): equal masses and equal Lambda give LambdaT = Lambda, dLambdaT = 0;
    LambdaT equals the mass-weighted definition (16/13) sum (X_a + 12 X_b) X_a^4 L_a."""
    one = np.ones(1)
    p = oracle.prepare(1.4 * one, 1.4 * one, 0 * one, 0 * one, 400 * one, 400 * one,
                       100 * one, np.zeros(1, np.uint8), 0 * one)
    assert abs(p["LamT"][0] - 400) < 1e-10 and abs(p["dLamT"][0]) < 1e-10
    assert abs(p["eta"][0] - 0.25) < 1e-15
    m1, m2, L1, L2 = 1.9, 1.2, 200.0, 900.0
    p = oracle.prepare(np.array([m2]), np.array([m1]), one * 0, one * 0, np.array([L2]),
                       np.array([L1]), one * 100, np.zeros(1, np.uint8), one * 0)
    M = m1 + m2
    X1, X2 = m1 / M, m2 / M
    lt = 16 / 13 * ((X1 + 12 * X2) * X1 ** 4 * L1 + (X2 + 12 * X1) * X2 ** 4 * L2)
    assert abs(p["LamT"][0] - lt) < 1e-10 * lt


def test_prepare_masses_and_redshift():
    """Sec. 2.1: detector-frame chirp mass and eta from (1+z) m with z = H0 dL / c;
    f_ISCO of the Sec. 2.2 footnote; tcoal in sidereal days."""
    m1, m2, dl = np.array([30.0]), np.array([20.0]), np.array([3000.0])
    p = oracle.prepare(m1, m2, np.array([0.5]), np.array([-0.2]), None, None, dl,
                       np.ones(1, np.uint8), np.array([0.25]))
    z = 70.0 * 3000.0 / 299792.458
    M = 50.0 * (1 + z)
    eta = 600.0 / 2500.0
    assert abs(p["eta"][0] - eta) < 1e-15
    assert abs(p["Mc"][0] - M * eta ** 0.6) < 1e-12 * M
    assert abs(p["dL"][0] - 3.0) < 1e-15
    assert abs(p["tc"][0] - 0.25 * 86164.0905) < 1e-9
    fisco = 1 / (6 ** 1.5 * math.pi * M * 4.925490947641267e-6)
    assert abs(p["fisco"][0] - fisco) < 1e-12 * fisco
    # m2 > m1 is reordered with its spin
    p = oracle.prepare(m2, m1, np.array([0.5]), np.array([-0.2]), None, None, dl,
                       np.zeros(1, np.uint8), np.array([0.0]))
    assert p["chi1z"][0] == -0.2 and p["chi2z"][0] == 0.5


def test_grid_rule():
    n = oracle.grid_npts(np.array([2.0, 2.0, 2.0]), np.array([10.0, 2.0e4, 2.1]), 40.0, 200, 20000)
    assert list(n) == [200, math.ceil(40 * math.log(1e4)), 200]


def test_grid_rule_at_integer_boundary():
    """ceil(40 ln(fmax/fmin)) for the doubles fmax next to 2 e^(369/40), where
    the argument is within 5e-14 of the integer 369: the oracle must follow the
    definition (a 200-bit evaluation decides), which double precision misses
    for arguments a few 1e-15 above the integer."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    f0 = float(2 * mpmath.exp(mpmath.mpf(369) / 40))
    fmax = [f0]
    for _ in range(6):
        fmax.insert(0, float(np.nextafter(fmax[0], -np.inf)))
        fmax.append(float(np.nextafter(fmax[-1], np.inf)))
    fmax = np.array(fmax)
    want = [int(mpmath.ceil(40 * mpmath.log(mpmath.mpf(f) / 2))) for f in fmax]
    got = oracle.grid_npts(np.full(len(fmax), 2.0), fmax, 40.0, 200, 20000)
    assert list(got) == want and 369 in want and 370 in want


# ---------------------------------------------------------------- antenna patterns
def test_antenna_tensor_equals_jks():
    """Pattern functions by tensor contraction equal the JKS closed form."""
    for _ in range(50):
        lat, L, gam = RNG.uniform(-1.5, 1.5), RNG.uniform(0, 6.3), RNG.uniform(0, 6.3)
        th, ph, ps = RNG.uniform(0, math.pi), RNG.uniform(0, 6.3), RNG.uniform(0, math.pi)
        zeta = RNG.choice([math.pi / 2, math.pi / 3])
        a = oracle.antenna(lat, L, gam, zeta, th, ph, ps)
        b = jks(lat, gam, zeta, th, ph, ps, L)
        assert abs(a[0] - b[0]) < 1e-14 and abs(a[1] - b[1]) < 1e-14


def test_triangle_arms_sum_to_zero_and_zenith_norm():
    """Closed triangle: the three arms' patterns sum to zero (Sec. 3.3).
    Source at the zenith of an L detector: F+^2 + Fx^2 = sin^2 zeta."""
    for _ in range(20):
        lat, L, gT = RNG.uniform(-1.5, 1.5), RNG.uniform(0, 6.3), RNG.uniform(0, 6.3)
        th, ph, ps = RNG.uniform(0, math.pi), RNG.uniform(0, 6.3), RNG.uniform(0, math.pi)
        arms = [oracle.antenna(lat, L, gT + math.pi / 6 + 2 * math.pi * k / 3, math.pi / 3,
                               th, ph, ps) for k in range(3)]
        assert abs(sum(a[0] for a in arms)) < 1e-15 and abs(sum(a[1] for a in arms)) < 1e-15
        fp, fx = oracle.antenna(lat, L, gT, math.pi / 2, math.pi / 2 - lat, L, ps)
        assert abs(fp * fp + fx * fx - 1.0) < 1e-14
        assert abs(oracle.antenna(lat, L, gT, math.pi / 2, th, ph, ps + math.pi / 2)[0]
                   + oracle.antenna(lat, L, gT, math.pi / 2, th, ph, ps)[0]) < 1e-14


# ---------------------------------------------------------------- strain: rotation and Doppler
def _one_event(cfg="c1", seed=11, zero_spin=False):
    cat, d, p = oracle_catalog(cfg, 1, seed=seed)
    ev = cat.ev[0].copy()
    if zero_spin:
        ev[9:13] = 0
    return ev, cat


def test_strain_rotation_follows_t_of_f():
    """|h(f)| = A(f) |F+(g) c+ + i Fx(g) cx| with Earth angle g = Omega_E (tc - tau*(f))."""
    ev, cat = _one_event("c1")
    det, psd, rot = gwcat.network("c1")
    f, h = oracle.strain(ev, 2.0, cat.fmax[0], 40, det[:1], 1)
    Mc, eta, dL, th, ph, io, ps, tc = ev[:8]
    row = det[0]
    for k in range(0, 40, 7):
        g = OMEGA_E * (tc - oracle.tau_star(Mc, eta, f[k]))
        A = amp0(Mc, dL) * f[k] ** (-7 / 6)
        for a in range(3):
            fp, fx = jks(row[0], row[2] + math.pi / 6 + 2 * math.pi * a / 3, math.pi / 3,
                         th, ph, ps, row[1] + g)
            q = A * abs(fp * (1 + math.cos(io) ** 2) / 2 + 1j * fx * math.cos(io))
            assert abs(abs(h[a, k]) - q) <= 1e-12 * q


def test_doppler_delay_between_sites():
    """Without rotation, arg(h1/h2) is linear in f with slope 2 pi (r1 - r2).n R_E / c."""
    ev, cat = _one_event("c0", zero_spin=True)
    d1 = [0.7, 0.2, 0.3, math.pi / 2, 0, 0]
    d2 = [-0.4, 2.1, 1.1, math.pi / 2, 0, 0]
    f, h1 = oracle.strain(ev, 10.0, 400.0, 64, np.array([d1]), 0)
    _, h2 = oracle.strain(ev, 10.0, 400.0, 64, np.array([d2]), 0)
    ph = np.unwrap(np.angle(h1[0] / h2[0]))
    slope = np.polyfit(f, ph, 1)[0]
    th, phi, tc = ev[3], ev[4], ev[7]
    g = OMEGA_E * tc
    n = np.array([math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])

    def r(lat, lon):
        L = lon + g
        return np.array([math.cos(lat) * math.cos(L), math.cos(lat) * math.sin(L), math.sin(lat)])

    expect = 2 * math.pi * (r(d1[0], d1[1]) - r(d2[0], d2[1])) @ n * R_EARTH / C_SI
    assert abs(slope - expect) < 1e-9 * abs(expect)


# ---------------------------------------------------------------- SNR quadrature
@pytest.mark.parametrize("p_exp", [0.0, -4.0, 2.0])
def test_snr_geometric_series_closed_form(p_exp):
    """Power-law PSD, leading-order amplitude, fixed antennas: the trapezoid sum on
    the geometric grid is a geometric series with a closed form; it also converges
    to the continuum integral (Sec. 3.2, SNR definition)."""
    ev, _ = _one_event("c0", zero_spin=True)
    det = np.array([[0.75, 0.17, 0.35, math.pi / 2, 0, 0]])
    psd = np.array([[10.0, 1e-49, 1, 1.0, 0, 0, 0, p_exp, 0, 0, 0]])
    fmin, fmax = 10.0, 900.0
    Mc, eta, dL, th, ph, io, ps, tc = ev[:8]
    fp, fx = jks(det[0, 0], det[0, 2], det[0, 3], th, ph, ps, det[0, 1] + OMEGA_E * tc)
    pol2 = abs(fp * (1 + math.cos(io) ** 2) / 2 + 1j * fx * math.cos(io)) ** 2
    K = 4 * amp0(Mc, dL) ** 2 * pol2 / (1e-49 * 10.0 ** (-p_exp))
    q = -7 / 3 - p_exp + 1            # exponent of f in w_k |h|^2 / S
    for n in (2, 7, 300):
        cat = oracle.Catalog(ev, 0, fmin, fmax, n)
        s, st = oracle.snr(cat, det, psd, 0)
        r = (fmax / fmin) ** (1 / (n - 1))
        rq = r ** q
        geo = sum(rq ** k for k in range(1, n - 1))
        total = fmin ** q * ((r - 1) / 2 + (r - 1 / r) / 2 * geo + (1 - 1 / r) / 2 * rq ** (n - 1))
        assert abs(s[0] ** 2 - K * total) <= 1e-13 * K * total
    cat = oracle.Catalog(ev, 0, fmin, fmax, 20000)
    s, _ = oracle.snr(cat, det, psd, 0)
    integral = K * (fmax ** q - fmin ** q) / q
    assert abs(s[0] ** 2 - integral) <= 2e-7 * integral


def test_closed_triangle_snr_does_not_depend_on_its_rotation():
    """The three arms' detector tensors sum to zero and are spaced by 120 deg:
    the sum of the arms' |h|^2 is invariant under a rotation of the triangle in
    its plane, so the SNR does not depend on gamma_T (with every arm on); with
    one arm off it does."""
    ev, _ = _one_event("c1")
    det = np.array([[0.7, 0.16, 0.0, math.pi / 3, 1, 0]])
    psd = np.array([[10.0, 1e-49, 3, 1.0, 2.0, 2.0, 0, -4.0, 0.0, 2.0, 0]])
    cat = oracle.Catalog(ev, 1, 2.0, 60.0, 120)
    base = oracle.snr(cat, det, psd, 1)[0][0]
    masked = oracle.Catalog(ev, 1, 2.0, 60.0, 120, np.uint32(0b110))
    mbase = oracle.snr(masked, det, psd, 1)[0][0]
    moved = []
    for gam in (0.3, 1.1, 2.5):
        d2 = det.copy()
        d2[0, 2] = gam
        assert abs(oracle.snr(cat, d2, psd, 1)[0][0] / base - 1) < 1e-13
        moved.append(abs(oracle.snr(masked, d2, psd, 1)[0][0] / mbase - 1))
    assert max(moved) > 1e-3


# ---------------------------------------------------------------- tabulated PSD
def test_psd_table_interpolation_pins():
    """Tabulated noise curves (Sec. 3.1, psd_path / is_ASD): log-log linear
    interpolation reproduces a power law exactly, gives the geometric mean at
    the logarithmic midpoint of two nodes and the node values at the nodes,
    squares an amplitude spectral density, multiplies by the row's scale, and
    is blind (infinite noise) outside the table; bad tables are refused."""
    f = np.geomspace(1.0, 1e4, 41)
    S = 3e-49 * (f / 10.0) ** -4.0
    oracle.set_psd_tables([(f, S, False), (f, np.sqrt(S), True),
                           (np.array([10.0, 100.0]), np.array([4e-48, 1e-50]), False)])
    rows = [oracle.table_row(0), oracle.table_row(1, 0.5), oracle.table_row(2)]
    for x in np.exp(RNG.uniform(0.0, math.log(1e4), 50)):
        want = 3e-49 * (x / 10.0) ** -4.0
        assert abs(oracle.psd_eval(rows, 0, x) / want - 1) < 1e-13
        assert abs(oracle.psd_eval(rows, 1, x) / (0.5 * want) - 1) < 1e-13
    mid = oracle.psd_eval(rows, 2, math.sqrt(1000.0))
    assert abs(mid / math.sqrt(4e-48 * 1e-50) - 1) < 1e-14
    assert abs(oracle.psd_eval(rows, 2, 10.0) / 4e-48 - 1) < 1e-15
    assert abs(oracle.psd_eval(rows, 2, 100.0) / 1e-50 - 1) < 1e-15
    assert math.isinf(oracle.psd_eval(rows, 2, 9.999)) and math.isinf(oracle.psd_eval(rows, 2, 100.01))
    for bad in ([1.0, 1.0], [2.0, 1.0]):
        with pytest.raises(ValueError):
            oracle.set_psd_tables([(np.array(bad), np.array([1.0, 1.0]), False)])
    with pytest.raises(ValueError):
        oracle.set_psd_tables([(np.array([1.0, 2.0]), np.array([1.0, 0.0]), False)])


def test_snr_with_psd_table_closed_forms():
    """SNR with a tabulated power law equals the SNR with the analytic power
    law; a table covering only part of the grid sums only the grid points
    inside it (trapezoid weights of the full grid), which for a power law is a
    partial geometric sum in closed form."""
    ev, _ = _one_event("c0", zero_spin=True)
    det = np.array([[0.75, 0.17, 0.35, math.pi / 2, 0, 0]])
    fmin, fmax, n = 10.0, 900.0, 300
    f = np.geomspace(1.0, 1e4, 21)
    oracle.set_psd_tables([(f, 3e-49 * (f / 10.0) ** -4.0, False),
                           (np.array([40.0, 200.0]), 3e-49 * (np.array([40.0, 200.0]) / 10.0) ** -4.0,
                            False)])
    cat = oracle.Catalog(ev, 0, fmin, fmax, n)
    s_an, _ = oracle.snr(cat, det, [[10.0, 3e-49, 1, 1.0, 0, 0, 0, -4.0, 0, 0, 0]], 0)
    s_tab, _ = oracle.snr(cat, det, [oracle.table_row(0)], 0)
    assert abs(s_tab[0] / s_an[0] - 1) < 1e-13
    s_part, _ = oracle.snr(cat, det, [oracle.table_row(1)], 0)
    Mc, eta, dL, th, ph, io, ps, tc = ev[:8]
    fp, fx = jks(det[0, 0], det[0, 2], det[0, 3], th, ph, ps, det[0, 1] + OMEGA_E * tc)
    pol2 = abs(fp * (1 + math.cos(io) ** 2) / 2 + 1j * fx * math.cos(io)) ** 2
    fk, wk = geom_grid(fmin, fmax, n)
    inside = (fk >= 40.0) & (fk <= 200.0)
    want = np.sum(4 * amp0(Mc, dL) ** 2 * pol2 * wk[inside] * fk[inside] ** (-7 / 3)
                  / (3e-49 * (fk[inside] / 10.0) ** -4.0))
    assert 0 < inside.sum() < n and abs(s_part[0] ** 2 / want - 1) < 1e-12


# ---------------------------------------------------------------- Fisher closed forms
def _fisher1(ev, pset, fmin, fmax, n, det, psd, rot, P):
    cat = oracle.Catalog(ev, pset, fmin, fmax, n)
    F, s, err, st = oracle.fisher(cat, det, psd, rot, P)
    assert st[0] == 0
    return F[0], s[0]


@pytest.mark.parametrize("rot", [0, 1])
def test_fisher_extrinsic_closed_forms(rot):
    """d h / d ln dL = -h gives dL^2 G_dLdL = SNR^2; d h/d Phic = -i h gives
    G_PhicPhic = SNR^2 and G_dL,Phic = 0.  Without rotation d h/d tc = 2 pi i f h
    gives G_tctc and G_tc,Phic in closed form."""
    ev, cat = _one_event("c1")
    det, psd, _ = gwcat.network("c1")
    n = 120
    F, s = _fisher1(ev, 1, 2.0, cat.fmax[0], n, det, psd, rot, 11)
    dL = ev[2]
    assert abs(dL ** 2 * F[2, 2] - s ** 2) < 1e-9 * s ** 2
    assert abs(F[8, 8] - s ** 2) < 1e-9 * s ** 2
    assert abs(F[2, 8]) < 1e-9 * math.sqrt(F[2, 2] * F[8, 8])
    if rot == 0:
        f, h = oracle.strain(ev, 2.0, cat.fmax[0], n, det, 0)
        fg, w = geom_grid(2.0, cat.fmax[0], n)
        W = 4 * w / psd_eval(psd[0], fg)
        m2 = (np.abs(h) ** 2).sum(axis=0)
        gtt = np.sum(W * (2 * math.pi * fg) ** 2 * m2)
        gtp = -np.sum(W * 2 * math.pi * fg * m2)
        assert abs(F[7, 7] - gtt) < 1e-9 * gtt
        assert abs(F[7, 8] - gtp) < 1e-9 * math.sqrt(F[7, 7] * F[8, 8])


def test_fisher_chirp_mass_closed_form():
    """Without spins, tides or rotation, Mc dPsi/dMc = f dPsi/df = -2 pi f tau*(f),
    so d h/d Mc = h (5/(6 Mc) - 2 pi i f tau*/Mc) and G_McMc, G_Mc,Phic follow."""
    ev, cat = _one_event("c0", zero_spin=True)
    det, psd, _ = gwcat.network("c0")
    n = 150
    F, s = _fisher1(ev, 0, 10.0, cat.fmax[0], n, det, psd, 0, 9)
    f, h = oracle.strain(ev, 10.0, cat.fmax[0], n, det, 0)
    fg, w = geom_grid(10.0, cat.fmax[0], n)
    W = 4 * w / psd_eval(psd[0], fg) * np.abs(h[0]) ** 2
    Mc, eta = ev[0], ev[1]
    tau = np.array([oracle.tau_star(Mc, eta, x) for x in fg])
    a = 5 / (6 * Mc)
    b = 2 * math.pi * fg * tau / Mc
    gmm = np.sum(W * (a ** 2 + b ** 2))
    gmp = np.sum(W * b)
    assert abs(F[0, 0] - gmm) < 1e-8 * gmm
    assert abs(F[0, 8] - gmp) < 1e-8 * math.sqrt(F[0, 0] * F[8, 8])
    assert abs(F[0, 2] - np.sum(W * a * (-1 / ev[2]))) < 1e-8 * math.sqrt(F[0, 0] * F[2, 2])


def test_fisher_iota_psi_closed_forms():
    """Without rotation the pattern functions are constant: d h/d iota and
    d h/d psi have closed forms through the JKS patterns."""
    ev, cat = _one_event("c0", zero_spin=True)
    det, psd, _ = gwcat.network("c0")
    n = 100
    F, s = _fisher1(ev, 0, 10.0, cat.fmax[0], n, det, psd, 0, 9)
    Mc, eta, dL, th, ph, io, ps, tc = ev[:8]
    row = det[0]
    fp, fx = jks(row[0], row[2], row[3], th, ph, ps, row[1] + OMEGA_E * tc)
    ci, si = math.cos(io), math.sin(io)
    cp = (1 + ci * ci) / 2
    fg, w = geom_grid(10.0, cat.fmax[0], n)
    K = np.sum(4 * w / psd_eval(psd[0], fg) * (amp0(Mc, dL) * fg ** (-7 / 6)) ** 2)
    d_io = fp * (-ci * si) + 1j * fx * (-si)
    d_ps = 2 * fx * cp - 2j * fp * ci
    q = fp * cp + 1j * fx * ci
    assert abs(s ** 2 - K * abs(q) ** 2) < 1e-12 * s ** 2
    assert abs(F[5, 5] - K * abs(d_io) ** 2) < 1e-9 * F[5, 5]
    assert abs(F[6, 6] - K * abs(d_ps) ** 2) < 1e-9 * F[6, 6]
    assert abs(F[5, 6] - K * (np.conj(d_io) * d_ps).real) < 1e-9 * math.sqrt(F[5, 5] * F[6, 6])


def test_fisher_symmetries():
    """SNR and Gamma are invariant under psi -> psi + pi and under a Phic shift;
    with rotation they are invariant under (tc, phi) -> (tc + D, phi + Omega_E D)."""
    ev, cat = _one_event("c1")
    det, psd, _ = gwcat.network("c1")
    n = 80
    F0, s0 = _fisher1(ev, 1, 2.0, cat.fmax[0], n, det, psd, 1, 11)
    scale = np.sqrt(np.outer(np.diag(F0), np.diag(F0)))
    for mod in ("psi", "phic", "tc"):
        e2 = ev.copy()
        if mod == "psi":
            e2[6] += math.pi
        elif mod == "phic":
            e2[8] += 1.3
        else:
            D = 5000.0
            e2[7] += D
            e2[4] += OMEGA_E * D
        F1, s1 = _fisher1(e2, 1, 2.0, cat.fmax[0], n, det, psd, 1, 11)
        assert abs(s1 - s0) < 1e-11 * s0
        assert np.max(np.abs(F1 - F0) / scale) < 1e-8


def test_fisher_step_insensitive():
    """The Richardson result does not depend on the first step (0.05-0.2 rad)."""
    cat, _, _ = oracle_catalog("c2", 2, max_npts=150)
    det, psd, rot = gwcat.network("c2")
    res = []
    for t in (0.05, 0.2):
        oracle.set_fd_target(t)
        F, s, err, st = oracle.fisher(cat, det, psd, rot, 11)
        res.append(F)
    oracle.set_fd_target(0.1)
    dg = np.sqrt(np.einsum("eii->ei", res[0]))
    rel = np.abs(res[1] - res[0]) / (dg[:, :, None] * dg[:, None, :])
    assert rel.max() < 5e-9


def test_config0_fisher_is_rank_five():
    """One detector with fixed patterns: dL, theta, phi, iota, psi, Phic enter
    through one complex amplitude, so the 9x9 Fisher has rank 5; the inversion
    flags every event (Sec. 4: condition number beyond the inverse precision)."""
    cat, _, _ = oracle_catalog("c0", 3, max_npts=120)
    det, psd, rot = gwcat.network("c0")
    F, s, err, st = oracle.fisher(cat, det, psd, rot, 9)
    for e in range(3):
        d = np.sqrt(np.diag(F[e]))
        lam = np.linalg.eigvalsh(F[e] / np.outer(d, d))
        assert np.sum(lam < 1e-9 * lam.max()) == 4
    C, k, eps, sti = oracle.invert(F)
    assert np.all((sti & (oracle.ST_ILL_COND | oracle.ST_NOT_PD)) != 0)


# ---------------------------------------------------------------- inversion
def test_invert_against_numpy():
    P = 11
    mats = []
    for _ in range(6):
        A = RNG.normal(size=(P, P))
        G = A @ A.T + P * np.eye(P)
        s = np.exp(RNG.uniform(-8, 8, P))
        mats.append(G * np.outer(s, s))
    F = np.array(mats)
    C, k, eps, st = oracle.invert(F)
    for e in range(len(F)):
        ref = np.linalg.inv(F[e])
        sc = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.max(np.abs(C[e] - ref) / sc) < 1e-12
        d = np.sqrt(np.diag(F[e]))
        lam = np.linalg.eigvalsh(F[e] / np.outer(d, d))
        assert abs(k[e] - lam.max() / lam.min()) < 1e-10 * k[e]
        assert st[e] == 0 and eps[e] < 1e-8
    bad = F[:3].copy()
    bad[0, 0, 1] = bad[0, 1, 0] = 10 * math.sqrt(bad[0, 0, 0] * bad[0, 1, 1])
    bad[1, 2, 2] = np.nan
    C, k, eps, st = oracle.invert(bad, cond_max=1e50)
    assert st[0] & oracle.ST_NOT_PD and np.isnan(C[0]).all()
    assert st[1] & oracle.ST_NONFINITE
    C, k, eps, st = oracle.invert(F[:1], cond_max=1.0)
    assert st[0] & oracle.ST_COND_GT_MAX and np.isnan(C[0]).all()


# ---------------------------------------------------------------- VJP references
def test_snr_grad_pins():
    """d SNR/d Phic = 0, d SNR/d dL = -SNR/dL; without rotation d SNR/d iota and
    d SNR/d psi follow from the JKS patterns."""
    ev, cat = _one_event("c0", zero_spin=True)
    det, psd, _ = gwcat.network("c0")
    n = 100
    c = oracle.Catalog(ev, 0, 10.0, cat.fmax[0], n)
    g = oracle.snr_grad(c, det, psd, 0, 9)[0]
    s, _ = oracle.snr(c, det, psd, 0)
    assert abs(g[8]) < 1e-10 * s[0]
    assert abs(g[2] + s[0] / ev[2]) < 1e-10 * abs(g[2])
    Mc, eta, dL, th, ph, io, ps, tc = ev[:8]
    row = det[0]
    fg, w = geom_grid(10.0, cat.fmax[0], n)
    K = math.sqrt(np.sum(4 * w / psd_eval(psd[0], fg) * (amp0(Mc, dL) * fg ** (-7 / 6)) ** 2))

    def snr_of(io_, ps_):
        fp, fx = jks(row[0], row[2], row[3], th, ph, ps_, row[1] + OMEGA_E * tc)
        return K * abs(fp * (1 + math.cos(io_) ** 2) / 2 + 1j * fx * math.cos(io_))

    fp, fx = jks(row[0], row[2], row[3], th, ph, ps, row[1] + OMEGA_E * tc)
    ci, si = math.cos(io), math.sin(io)
    q = fp * (1 + ci * ci) / 2 + 1j * fx * ci
    dq_io = fp * (-ci * si) + 1j * fx * (-si)
    dq_ps = 2 * fx * (1 + ci * ci) / 2 - 2j * fp * ci
    assert abs(snr_of(io, ps) - s[0]) < 1e-12 * s[0]
    assert abs(g[5] - K * (np.conj(q) * dq_io).real / abs(q)) < 1e-9 * s[0]
    assert abs(g[6] - K * (np.conj(q) * dq_ps).real / abs(q)) < 1e-9 * s[0]


def test_logdet_grad_gamma_matches_jacobi_formula():
    """d log det Gamma / d gamma = tr(Gamma^-1 d Gamma/d gamma) (Jacobi's formula),
    with d Gamma/d gamma from differences of whole Fisher matrices; the oracle
    differences log det itself.  Tidal BNS on the five-interferometer network
    (well conditioned enough for an elementwise difference of Gamma)."""
    cat, _, _ = oracle_catalog("c2", 1, max_npts=60)
    det, psd, rot = gwcat.network("c4")
    gg, ldet = oracle.logdet_grad_gamma(cat, det, psd, rot, 11, [1, 2])
    F0, s0, _, _ = oracle.fisher(cat, det, psd, rot, 11)
    Finv = np.linalg.inv(F0[0])
    d = np.sqrt(np.diag(F0[0]))
    sign, v = np.linalg.slogdet(F0[0] / np.outer(d, d))
    assert sign > 0 and abs(v + 2 * np.sum(np.log(d)) - ldet[0]) < 1e-8 * abs(ldet[0])
    for q, di in enumerate([1, 2]):
        def fisher_at(gam):
            d2 = det.copy()
            d2[di, 2] = gam
            return oracle.fisher(cat, d2, psd, rot, 11)[0][0]
        h = 0.02
        dG = (8 * (fisher_at(det[di, 2] + h) - fisher_at(det[di, 2] - h))
              - (fisher_at(det[di, 2] + 2 * h) - fisher_at(det[di, 2] - 2 * h))) / (12 * h)
        jac = np.trace(Finv @ dG)
        assert abs(gg[q] - jac) < 1e-4 * (abs(jac) + 1)


# ---------------------------------------------------------------- duty factor
def _masked(cat, masks):
    return oracle.Catalog(cat.ev, cat.pset, cat.fmin, cat.fmax, cat.npts, masks)


def test_arm_masks_snr_is_quadrature_sum_of_on_arms():
    """Duty factor (Sec. 3.2; the duty_factor option of Sec. 5, applied to every
    detector and to each arm of a triangle): the network SNR^2 of an event is the
    sum of the SNR^2 of the arms that are on (Eq. (3.2)); the per-arm SNR of an
    arm that is on does not depend on the others; no arm on gives zero."""
    cat, _, _ = oracle_catalog("c4", 6, seed=31, max_npts=150)
    det, psd, rot = gwcat.network("c4")
    na = oracle.n_arms(det)
    assert na == 5
    s0, arm0, _ = oracle.snr(cat, det, psd, rot, per_arm=True)
    masks = np.array([0b11111, 0b00001, 0b00110, 0b11000, 0, 0b10101], dtype=np.uint32)
    s1, arm1, st1 = oracle.snr(_masked(cat, masks), det, psd, rot, per_arm=True)
    assert (st1 == 0).all()
    for e in range(len(masks)):
        on = [(int(masks[e]) >> a) & 1 for a in range(na)]
        expect2 = sum(arm0[e, a] ** 2 for a in range(na) if on[a])
        assert abs(s1[e] ** 2 - expect2) <= 1e-13 * s0[e] ** 2
        for a in range(na):
            assert arm1[e, a] == (arm0[e, a] if on[a] else 0.0)
    assert s1[0] == s0[0] and s1[4] == 0.0


@pytest.mark.parametrize("k", [0, 1, 2])
def test_masked_triangle_arm_equals_standalone_interferometer(k):
    """A triangle is three co-located 60-degree interferometers (Sec. 3.3): with
    only arm k on, SNR and Fisher equal those of a network that holds just an
    L-shaped detector of opening 60 degrees at bisector gamma_T + 30 + 120 k deg."""
    cat, _, _ = oracle_catalog("c1", 2, seed=5, max_npts=120)
    det, psd, rot = gwcat.network("c1")
    tri = det[0]
    F1, s1, _, st1 = oracle.fisher(_masked(cat, np.uint32(1 << k)), det, psd, rot, 11)
    solo = np.array([[tri[0], tri[1], tri[2] + math.pi / 6 + 2 * math.pi * k / 3, math.pi / 3,
                      0, tri[5]]])
    F2, s2, _, st2 = oracle.fisher(cat, solo, psd, rot, 11)
    assert (st1 == 0).all() and (st2 == 0).all()
    np.testing.assert_allclose(s1, s2, rtol=1e-13)
    for e in range(2):
        sc = np.sqrt(np.outer(np.diag(F2[e]), np.diag(F2[e])))
        assert np.max(np.abs(F1[e] - F2[e]) / sc) < 1e-9


def test_fisher_additive_over_disjoint_arm_sets():
    """Gamma is a sum over detectors and arms (Eq. (3.3)): for disjoint arm sets A
    and B, Gamma(A u B) = Gamma(A) + Gamma(B) (to the finite-difference error bar,
    as each set picks its own steps); with no arm on Gamma = 0 and SNR = 0."""
    cat, _, _ = oracle_catalog("c4", 3, seed=41, max_npts=120)
    det, psd, rot = gwcat.network("c4")
    FA, sA, _, _ = oracle.fisher(_masked(cat, np.uint32(0b00101)), det, psd, rot, 11)
    FB, sB, _, _ = oracle.fisher(_masked(cat, np.uint32(0b11010)), det, psd, rot, 11)
    F, s, _, _ = oracle.fisher(cat, det, psd, rot, 11)
    F0, s0, _, st0 = oracle.fisher(_masked(cat, np.uint32(0)), det, psd, rot, 11)
    np.testing.assert_allclose(sA ** 2 + sB ** 2, s ** 2, rtol=1e-13)
    for e in range(3):
        sc = np.sqrt(np.outer(np.diag(F[e]), np.diag(F[e])))
        assert np.max(np.abs(FA[e] + FB[e] - F[e]) / sc) < 1e-8
    assert (st0 == 0).all() and (F0 == 0).all() and (s0 == 0).all()


def test_masked_snr_gradient_closed_forms():
    """With any set of arms on, h is proportional to 1/dL, so d SNR / d dL = -SNR/dL;
    SNR does not depend on Phic (h -> h e^{-i dPhic})."""
    cat, _, _ = oracle_catalog("c4", 2, seed=43, max_npts=100)
    det, psd, rot = gwcat.network("c4")
    masks = np.array([0b01010, 0b10001], dtype=np.uint32)
    mc = _masked(cat, masks)
    g = oracle.snr_grad(mc, det, psd, rot, 11)
    s, _ = oracle.snr(mc, det, psd, rot)
    np.testing.assert_allclose(g[:, 2], -s / cat.ev[:, 2], rtol=1e-9)
    assert np.all(np.abs(g[:, 8]) <= 1e-9 * s)


def test_masked_off_detector_has_no_orientation_gradient():
    """A detector that is off for every event contributes nothing to any Fisher
    matrix, so d(sum log det Gamma)/d gamma of that detector is exactly zero,
    while the detectors that are on keep their gradient."""
    cat, _, _ = oracle_catalog("c4", 2, seed=47, max_npts=100)
    det, psd, rot = gwcat.network("c4")
    mc = _masked(cat, np.uint32(0b01111))          # triangle + first L on, second L off
    g, ldet = oracle.logdet_grad_gamma(mc, det, psd, rot, 11, [1, 2])
    assert np.isfinite(ldet).all()
    assert g[1] == 0.0 and g[0] != 0.0


def test_snr_gate_selection_brute_force():
    """The detection gate (Sec. 5, snr_th) keeps exactly the events with SNR above
    the threshold, in catalog order; NaN (flagged) events and SNR == threshold
    are dropped.  Checked against a plain loop."""
    rng = np.random.default_rng(3)
    snr = rng.uniform(0, 30, 500)
    snr[::37] = np.nan
    snr[5] = 12.0
    idx = oracle.select_snr(snr, 12.0)
    brute = [e for e in range(len(snr)) if snr[e] == snr[e] and snr[e] > 12.0]
    assert idx.tolist() == brute and idx.dtype == np.int64
    assert oracle.select_snr(np.array([]), 1.0).size == 0


# ---------------------------------------------------------------- covariance tools
def _spd(P, kappa_log10, rng):
    """Random symmetric positive-definite matrix with a spread of eigenvalues and
    a non-trivial diagonal scale."""
    Q, _ = np.linalg.qr(rng.normal(size=(P, P)))
    w = 10.0 ** np.linspace(0, -kappa_log10, P)
    D = np.diag(10.0 ** rng.uniform(-3, 3, P))
    return D @ (Q * w) @ Q.T @ D


def test_fisher_eig_matches_library_and_residuals():
    """CheckFisher (Sec. 4.1): eigenvalues equal LAPACK's (numpy.linalg.eigvalsh) on
    the normalised matrix; A V = V diag(w) with V orthonormal."""
    rng = np.random.default_rng(21)
    F = np.stack([_spd(11, 6, rng) for _ in range(4)])
    w, V = oracle.fisher_eig(F, normalize=True)
    for e in range(4):
        d = np.sqrt(np.diag(F[e]))
        A = F[e] / np.outer(d, d)
        np.testing.assert_allclose(w[e], np.linalg.eigvalsh(A), rtol=1e-9, atol=1e-14)
        assert np.max(np.abs(A @ V[e] - V[e] * w[e])) < 1e-13
        assert np.max(np.abs(V[e].T @ V[e] - np.eye(11))) < 1e-13
    w2, _ = oracle.fisher_eig(F, normalize=False)
    np.testing.assert_allclose(w2[0], np.linalg.eigvalsh(F[0]), rtol=1e-8, atol=1e-12 * np.abs(w2[0]).max())


@pytest.mark.parametrize("method", range(6))
def test_covariance_methods_agree_with_library_inverse(method):
    """Every inversion method of CovMatr (Sec. 4.1) gives the inverse of a
    positive-definite matrix; the normalisation is undone; eps = max|G C - 1|."""
    rng = np.random.default_rng(22)
    F = np.stack([_spd(11, 5, rng) for _ in range(3)])
    C, k, eps, st = oracle.covariance(F, method=method)
    assert (st == 0).all()
    for e in range(3):
        Cn = np.linalg.inv(F[e])
        sc = np.sqrt(np.outer(np.diag(Cn), np.diag(Cn)))
        assert np.max(np.abs(C[e] - Cn) / sc) < 1e-9
        # eps of the double-rounded C: diagonal scales of 1e+-3 amplify its rounding
        assert eps[e] < 1e-6
        R = F[e].astype(np.longdouble) @ C[e].astype(np.longdouble) - np.eye(11)
        assert abs(eps[e] - float(np.max(np.abs(R)))) < 1e-6 * eps[e]
        d = np.sqrt(np.diag(F[e]))
        wn = np.linalg.eigvalsh(F[e] / np.outer(d, d))
        assert abs(k[e] / (wn[-1] / wn[0]) - 1) < 1e-6


def test_covariance_svd_truncation_closed_forms():
    """Truncated SVD and svd_reg (Sec. 4.1) on a matrix with unit diagonal, a 2x2
    block [[1, c], [c, 1]] with c = 1 - 2^-52 (singular values 2 - 2^-52 and 2^-52,
    ratio below the 1e-15 threshold) and the identity elsewhere.  Truncation
    replaces 2^-52 by 1e-15 s_max; svd_reg drops it."""
    P = 11
    c = 1.0 - 2.0 ** -52
    F = np.eye(P)
    F[0, 1] = F[1, 0] = c
    s1, s2 = 1.0 + c, 1.0 - c
    assert s2 == 2.0 ** -52
    v1 = np.array([1.0, 1.0]) / math.sqrt(2)
    v2 = np.array([1.0, -1.0]) / math.sqrt(2)
    C3, k3, _, st3 = oracle.covariance(F[None], method=oracle.INV_SVD_TRUNC, thresh=1e-15)
    want3 = np.outer(v1, v1) / s1 + np.outer(v2, v2) / (1e-15 * s1)
    np.testing.assert_allclose(C3[0, :2, :2], want3, rtol=1e-12)
    C4, _, _, st4 = oracle.covariance(F[None], method=oracle.INV_SVD_REG, thresh=1e-15)
    np.testing.assert_allclose(C4[0, :2, :2], np.outer(v1, v1) / s1, rtol=1e-12)
    np.testing.assert_allclose(C4[0, 2:, 2:], np.eye(P - 2), rtol=1e-15)
    assert abs(k3[0] / (s1 / s2) - 1) < 1e-3      # 2^-52 from a long-double Jacobi sweep
    assert (st3 & oracle.ST_ILL_COND).all() and (st4 & oracle.ST_ILL_COND).all()


def test_covariance_fix_prior_and_marginalisation_identities():
    """fixParams = inverse of the kept block; marginalising = taking the block of
    the full inverse, which equals the inverse of the Schur complement; addPrior =
    inverse of Gamma + diag(prior), and a very tight prior approaches fixing."""
    rng = np.random.default_rng(23)
    F = np.stack([_spd(11, 4, rng) for _ in range(2)])
    keep = [0, 1, 2, 3, 5, 7, 8]
    drop = [4, 6, 9, 10]
    Cf, _, _, st = oracle.covariance(F, keep=keep, method=oracle.INV_CHO)
    Cfull, _, _, _ = oracle.covariance(F, method=oracle.INV_CHO)
    prior = np.zeros(11)
    prior[[4, 6]] = [3.0e2, 5.0e-1]
    Cp, _, _, _ = oracle.covariance(F, prior=prior, method=oracle.INV_CHO)
    big = np.zeros(11)
    big[drop] = 1e30
    Cb, _, _, _ = oracle.covariance(F, prior=big, method=oracle.INV_SVD)
    for e in range(2):
        A = F[e][np.ix_(keep, keep)]
        np.testing.assert_allclose(Cf[e], np.linalg.inv(A), rtol=1e-9)
        schur = A - F[e][np.ix_(keep, drop)] @ np.linalg.solve(F[e][np.ix_(drop, drop)],
                                                               F[e][np.ix_(drop, keep)])
        np.testing.assert_allclose(Cfull[e][np.ix_(keep, keep)], np.linalg.inv(schur), rtol=1e-8)
        np.testing.assert_allclose(Cp[e], np.linalg.inv(F[e] + np.diag(prior)), rtol=1e-9)
        np.testing.assert_allclose(Cb[e][np.ix_(keep, keep)], Cf[e], rtol=1e-8)


def test_covariance_not_pd_fallbacks_and_cond_max():
    """A symmetric indefinite matrix: Cholesky fails (NaN, status NOT_PD); the
    default falls back to the SVD (status bit 128) and LU inverts it, both equal
    to the library inverse; above cond_max nothing is inverted."""
    rng = np.random.default_rng(24)
    Q, _ = np.linalg.qr(rng.normal(size=(9, 9)))
    F = ((Q * np.array([3, 2, 1.5, 1, 0.7, 0.5, -0.4, 0.3, 0.2])) @ Q.T)[None]
    C0, _, _, st0 = oracle.covariance(F, method=oracle.INV_CHO)
    assert st0[0] & oracle.ST_NOT_PD and np.isnan(C0).all()
    want = np.linalg.inv(F[0])
    for m, bit in ((oracle.INV_CHO_SVD, oracle.ST_SVD_FALLBACK), (oracle.INV_LU, 0)):
        C, _, eps, st = oracle.covariance(F, method=m)
        np.testing.assert_allclose(C[0], want, rtol=1e-9, atol=1e-12)
        assert (st[0] & oracle.ST_SVD_FALLBACK) == bit and eps[0] < 1e-9
    G = np.stack([_spd(11, 8, rng)])
    C, k, _, st = oracle.covariance(G, cond_max=1e5)
    assert st[0] & oracle.ST_COND_GT_MAX and np.isnan(C).all() and k[0] > 1e5


def test_sky_area_is_the_gaussian_confidence_ellipse():
    """Delta Omega_X (Sec. 4.1): for a Gaussian in (theta, phi) with covariance C,
    the ellipse x^T C^-1 x <= k of solid angle Delta Omega = |sin theta| pi k
    sqrt(det C) holds a fraction X of the probability (Monte Carlo, 2e6 draws)."""
    rng = np.random.default_rng(25)
    theta = 1.1
    Cang = np.array([[4e-4, -1.5e-4], [-1.5e-4, 2.5e-4]])
    C = np.eye(11) * 1e-2
    C[3:5, 3:5] = Cang
    for X in (50.0, 90.0):
        a_sr = oracle.sky_area(C[None], 3, 4, [theta], perc=X, units="Sterad")[0]
        a_dg = oracle.sky_area(C[None], 3, 4, [theta], perc=X, units="SqDeg")[0]
        assert abs(a_dg / a_sr - (180 / math.pi) ** 2) < 1e-12 * a_dg / a_sr
        k = a_sr / (abs(math.sin(theta)) * math.pi * math.sqrt(np.linalg.det(Cang)))
        x = rng.multivariate_normal([0, 0], Cang, size=2_000_000)
        q = np.einsum("ni,ij,nj->n", x, np.linalg.inv(Cang), x)
        frac = np.mean(q <= k)
        assert abs(frac - X / 100) < 2e-3, (X, frac)


# ---------------------------------------------------------------- Table 2 fixture
def _table2():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "detectors_table2.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, lat, lon, gam, zeta, shape = line.split()
            rows[name] = (float(lat), float(lon), float(gam), float(zeta), shape)
    return rows


def test_table2_triangle_is_the_configs_triangle():
    """The synthetic networks' triangle is the ET Sardinia row of Table 2."""
    lat, lon, gam, zeta, shape = _table2()["ETS"]
    D = math.pi / 180
    assert shape == "T"
    np.testing.assert_allclose(gwcat.DET_TRI[:4], [lat * D, lon * D, gam * D, zeta * D], rtol=1e-15)
    assert gwcat.DET_TRI[4] == 1


def test_table2_hanford_livingston_delay():
    """Table 2's H1 and L1 positions: for a source along the baseline the strain
    phase difference grows as 2 pi f |r_H - r_L| / c (about 10 ms of light travel
    between the sites); for a source perpendicular to it, as 0."""
    t = _table2()
    D = math.pi / 180
    ev, _ = _one_event("c0", zero_spin=True)
    g = OMEGA_E * ev[7]

    def rvec(name):
        lat, lon = t[name][0] * D, t[name][1] * D + g
        return np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])

    b = (rvec("H1") - rvec("L1")) * R_EARTH
    dets = [np.array([[t[k][0] * D, t[k][1] * D, t[k][2] * D, t[k][3] * D, 0, 0]]) for k in ("H1", "L1")]
    for n, want in ((b / np.linalg.norm(b), np.linalg.norm(b) / C_SI), (None, 0.0)):
        if n is None:   # a direction perpendicular to the baseline
            n = np.cross(b, [0.0, 0.0, 1.0])
            n /= np.linalg.norm(n)
        e2 = ev.copy()
        e2[3] = math.acos(n[2])
        e2[4] = math.atan2(n[1], n[0])
        f, hH = oracle.strain(e2, 10.0, 400.0, 64, dets[0], 0)
        _, hL = oracle.strain(e2, 10.0, 400.0, 64, dets[1], 0)
        slope = np.polyfit(f, np.unwrap(np.angle(hH[0] / hL[0])), 1)[0]
        assert abs(slope / (2 * math.pi) - want) < 1e-9 * max(want, 1e-3)
    assert 9.9e-3 < np.linalg.norm(b) / C_SI < 1.01e-2


def test_perturb_fisher_definition():
    """perturb_Fisher (Sec. 4.1): symmetric relative perturbation at the eps-th
    decimal; eps = 0 returns the input; |Gamma' - Gamma| <= eps |Gamma|."""
    rng = np.random.default_rng(26)
    F = np.stack([_spd(11, 4, rng) for _ in range(3)])
    F = 0.5 * (F + np.transpose(F, (0, 2, 1)))
    r = rng.uniform(-1, 1, F.shape)
    Fp = oracle.perturb_fisher(F, r, 1e-10)
    assert np.array_equal(oracle.perturb_fisher(F, r, 0.0), F)
    assert np.array_equal(Fp, np.transpose(Fp, (0, 2, 1)))
    assert np.all(np.abs(Fp - F) <= 1e-10 * np.abs(F) * (1 + 1e-15))
    i, j = 2, 7
    assert Fp[1, i, j] == F[1, i, j] * (1.0 + 1e-10 * r[1, i, j])
