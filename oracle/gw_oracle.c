/*
 * gw_oracle.c -- plain, slow, single-threaded CPU oracle for the Fisher-forecast
 * hot path of GWFAST (arXiv:2207.06910).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg, and by
 * nothing else.  It shares no code, header, table or constant generator with the
 * CUDA library; neither side includes or links the other.
 *
 * Arithmetic: long double everywhere (80-bit on x86-64, binary128 on aarch64);
 * results are returned as double.  Every parameter derivative is taken by
 * Richardson-extrapolated central differences of the full complex strain
 * h(f) = Q(f) exp(i Phi(f)); nothing is differentiated by hand.
 *
 * What each function follows (paper = arXiv:2207.06910):
 *   or_prepare ......... Sec. 2.1 (parameters, Table 1; Lambda-tilde and
 *                        delta-Lambda-tilde, Eq. (2.2)); f_ISCO, Sec. 2.2 footnote.
 *   or_psi_pn .......... TaylorF2 3.5PN phase (Sec. 2.2, Buonanno et al. 2009),
 *                        spin-orbit (1.5PN) and spin-spin (2PN) leading terms,
 *                        5PN+6PN tidal terms in the Lambda-tilde form (Wade et al.
 *                        2014, cited in Sec. 2.1).
 *   or_tau_star ........ time to coalescence, 3.5PN (Sec. 2.2 footnote: Buonanno
 *                        et al. 2009 Eq. (3.8b)).
 *   or_antenna ......... pattern functions as the contraction D^{ij} e^A_{ij}
 *                        of the detector tensor with the polarisation tensors
 *                        (Sec. 3.1, with Earth rotation along t(f)).
 *   or_strain .......... detector strain with Earth-rotation Doppler phase
 *                        (Sec. 3.1 footnote on Earth motion).
 *   or_set_psd_tables .. tabulated noise curves (Sec. 3.1, psd_path / is_ASD),
 *                        log-log linear interpolation.
 *   or_snr ............. SNR_i^2 = 4 int |h|^2/S_n df; network sum in quadrature
 *                        (Sec. 3.2, Eqs. (3.1)-(3.2)); trapezoid on the log grid.
 *                        SNR, Fisher and the two VJP references take optional
 *                        per-event arm masks: the duty factor (Sec. 3.2, and the
 *                        duty_factor option of Sec. 5), applied to each detector
 *                        and to each arm of a triangle separately.
 *   or_fisher .......... Gamma_ij = 4 int Re(d_i h d_j h*)/S_n df, summed over
 *                        detectors and triangle arms (Sec. 3.2, Eq. (3.3)).
 *   or_invert .......... normalise by sqrt(diag), Cholesky inverse, condition
 *                        number from eigenvalues, inversion error
 *                        eps = max|Gamma Gamma^-1 - 1| (Sec. 4.1).
 *   or_snr_grad ........ d SNR / d theta_i by Richardson differences of SNR.
 *   or_logdet_grad_gamma d (sum_e log det Gamma_e) / d gamma_d by Richardson
 *                        differences over the detector orientation.
 *   or_fisher_eig ...... eigenvalues / eigenvectors of the (normalised) Fisher
 *                        matrix (CheckFisher, Sec. 4.1), cyclic Jacobi.
 *   or_covariance ...... CovMatr with its inversion methods (Cholesky, Cholesky
 *                        with SVD fallback, SVD, truncated SVD, svd_reg, LU),
 *                        fixParams and addPrior (Secs. 4.1-4.2).
 *   or_sky_area ........ Delta Omega_X% (Sec. 4.1, the localisation formula).
 *
 * Conventions (the paper gives none of these formulas; they are fixed here):
 *   h = Q exp(i Phi),  Q = A [F+ (1+cos^2 iota)/2 + i Fx cos iota],
 *   Phi = 2 pi f (tc - tc_fid) - Phic - pi/4 + Psi_PN + Psi_tidal + Phi_D,
 *   Phi_D = 2 pi f (R_E/c) rhat_det . nhat,   t(f) = tc - tau*(f),
 *   Earth angle g(f) = Omega_E t(f) (rotation on) or Omega_E tc_fid (off).
 *   Detector arms at gamma -/+ zeta/2 from local East (counter-clockwise),
 *   D = (u u^T - w w^T)/2; p = cos(psi) e_phi + sin(psi) e_theta,
 *   q = -sin(psi) e_phi + cos(psi) e_theta, e+ = pp^T - qq^T, ex = pq^T + qp^T.
 *   A triangle is three co-located 60-degree interferometers with bisectors
 *   gamma_T + 30 deg + 120 deg k, k = 0,1,2.
 *
 * Parity pins: see tests/test_oracle_pins.py.  Parity unpinned here: none of
 * the functions; the spin terms are pinned only through the equivalent
 * (chi_s, chi_a) form.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double ld;
typedef long double _Complex cld;

#define OR_PI 3.141592653589793238462643383279502884L
#define OR_EULER_GAMMA 0.577215664901532860606512090082402431L

static const ld OR_TSUN = 4.925490947641267e-6L;     /* G Msun / c^3  [s]   */
static const ld OR_C = 299792458.0L;                 /* [m/s]               */
static const ld OR_MPC = 3.085677581491367e22L;      /* [m]                 */
static const ld OR_REARTH = 6.371e6L;                /* [m]                 */
static const ld OR_TSID = 86164.0905L;               /* sidereal day [s]    */
static const ld OR_H0 = 70.0L;                       /* km/s/Mpc            */
static const ld OR_CKMS = 299792.458L;               /* [km/s]              */

/* parameter slots of the full waveform parameter vector */
enum { I_MC, I_ETA, I_DL, I_TH, I_PH, I_IOTA, I_PSI, I_TC, I_PHIC,
       I_CHI1, I_CHI2, I_LT, I_DLT, N_ALL };

/* status bits (shared meaning with the library, defined independently) */
enum { ST_NOT_PD = 1, ST_COND_GT_MAX = 2, ST_NONFINITE = 4, ST_EMPTY_GRID = 8,
       ST_BAD_PARAM = 16, ST_ILL_COND = 32, ST_SVD_FALLBACK = 128 };

/* ------------------------------------------------------------------ */
/* detector table: per detector 6 doubles  lat, lon, gamma, zeta, shape, psd  */
/* psd table: per psd 11 doubles  f0, scale, nterm, c0..c3, p0..p3              */
typedef struct { ld lat, lon, gam, zeta; int psd; } arm_t;

static int expand_arms(int ndet, const double *det, arm_t *arms, int maxarms)
{
    int na = 0;
    for (int d = 0; d < ndet; d++) {
        const double *q = det + 6 * d;
        int shape = (int)q[4];
        if (shape == 0) {
            if (na >= maxarms) return -1;
            arms[na].lat = q[0]; arms[na].lon = q[1]; arms[na].gam = q[2];
            arms[na].zeta = q[3]; arms[na].psd = (int)q[5]; na++;
        } else {
            for (int k = 0; k < 3; k++) {
                if (na >= maxarms) return -1;
                arms[na].lat = q[0]; arms[na].lon = q[1];
                arms[na].gam = (ld)q[2] + OR_PI / 6 + 2 * OR_PI * k / 3;
                arms[na].zeta = OR_PI / 3; arms[na].psd = (int)q[5]; na++;
            }
        }
    }
    return na;
}

/* Duty factor (Sec. 3.2 and the duty_factor option of Sec. 5): each detector,
 * and each arm of a triangle separately, is on or off for a whole event.  The
 * arms of event e that are on are the bits of arm_mask[e] (bit a = arm a of
 * the expanded list above); arm_mask == NULL means every arm is on.  The
 * random draws are made by the caller and passed in.                       */
static int select_arms(const arm_t *all, int na, const uint32_t *arm_mask, int64_t e, arm_t *out)
{
    int m = 0;
    for (int a = 0; a < na; a++)
        if (!arm_mask || ((arm_mask[e] >> a) & 1u)) out[m++] = all[a];
    return m;
}

/* Tabulated noise curves (the psd_path / is_ASD detector options of Sec. 3.1):
 * a PSD row whose term count is -(k+1) reads table k, given as frequencies f_j
 * (strictly increasing, > 0) and values S_j (> 0; amplitude spectral density
 * when is_asd, squared here).  S_n(f) is the straight line through
 * (ln f_j, ln S_j) and (ln f_{j+1}, ln S_{j+1}) for f_j <= f <= f_{j+1}, times
 * the row's scale; outside [f_0, f_last] the detector is blind (S_n infinite,
 * zero weight). */
#define OR_MAX_TAB 8
static int g_ntab = 0;
static int64_t g_tab_n[OR_MAX_TAB];
static ld *g_tab_lnf[OR_MAX_TAB], *g_tab_lns[OR_MAX_TAB];

int or_set_psd_tables(int ntab, const int64_t *n, const double *f, const double *s,
                      const int32_t *is_asd)
{
    for (int k = 0; k < g_ntab; k++) { free(g_tab_lnf[k]); free(g_tab_lns[k]); }
    g_ntab = 0;
    if (ntab < 0 || ntab > OR_MAX_TAB) return 1;
    int64_t o = 0;
    for (int k = 0; k < ntab; k++) {          /* check every table first */
        if (n[k] < 2) return 1;
        for (int64_t j = 0; j < n[k]; j++)
            if (!(f[o + j] > 0) || !(s[o + j] > 0) || (j > 0 && !(f[o + j] > f[o + j - 1])))
                return 1;
        o += n[k];
    }
    o = 0;
    for (int k = 0; k < ntab; k++) {
        g_tab_lnf[k] = malloc(sizeof(ld) * n[k]);
        g_tab_lns[k] = malloc(sizeof(ld) * n[k]);
        g_tab_n[k] = n[k];
        for (int64_t j = 0; j < n[k]; j++) {
            g_tab_lnf[k][j] = logl((ld)f[o + j]);
            g_tab_lns[k][j] = (is_asd && is_asd[k] ? 2.0L : 1.0L) * logl((ld)s[o + j]);
        }
        o += n[k];
    }
    g_ntab = ntab;
    return 0;
}

static ld psd_table(int k, ld f)
{
    const ld x = logl(f);
    const ld *lf = g_tab_lnf[k], *ls = g_tab_lns[k];
    const int64_t n = g_tab_n[k];
    if (x < lf[0] || x > lf[n - 1]) return INFINITY;
    int64_t lo = 0, hi = n - 1;            /* lf[lo] <= x <= lf[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (lf[mid] <= x) lo = mid;
        else hi = mid;
    }
    return expl(ls[lo] + (ls[hi] - ls[lo]) * (x - lf[lo]) / (lf[hi] - lf[lo]));
}

static ld psd_eval(const double *psd, int idx, ld f)
{
    const double *q = psd + 11 * idx;
    ld s = 0;
    int nt = (int)q[2];
    if (nt < 0) {
        int k = -nt - 1;
        return k < g_ntab ? (ld)q[1] * psd_table(k, f) : NAN;
    }
    for (int j = 0; j < nt; j++) s += (ld)q[3 + j] * powl(f / (ld)q[0], (ld)q[7 + j]);
    return (ld)q[1] * s;
}

/* S_n(f) of PSD row idx (exported for the pins) */
double or_psd_eval(const double *psd, int idx, double f) { return (double)psd_eval(psd, idx, f); }

/* ------------------------------------------------------------------ */
/* TaylorF2 phase (restricted PN), all masses in seconds                */
static ld psi_pn_l(ld Mc_s, ld eta, ld chi1, ld chi2, ld LT, ld dLT, ld f)
{
    const ld pi = OR_PI, pi2 = OR_PI * OR_PI;
    ld M = Mc_s * powl(eta, -0.6L);
    ld v = cbrtl(pi * M * f);
    ld d = sqrtl(fmaxl(0.0L, 1.0L - 4.0L * eta));
    ld X1 = 0.5L * (1.0L + d), X2 = 0.5L * (1.0L - d);
    ld beta = (113.0L / 12.0L * X1 * X1 + 25.0L * eta / 4.0L) * chi1
            + (113.0L / 12.0L * X2 * X2 + 25.0L * eta / 4.0L) * chi2;
    ld sigma = 79.0L / 8.0L * eta * chi1 * chi2;
    ld vlso = 1.0L / sqrtl(6.0L);
    ld ph[8];
    ph[0] = 1.0L;
    ph[1] = 0.0L;
    ph[2] = 3715.0L / 756.0L + 55.0L / 9.0L * eta;
    ph[3] = -16.0L * pi + 4.0L * beta;
    ph[4] = 15293365.0L / 508032.0L + 27145.0L / 504.0L * eta + 3085.0L / 72.0L * eta * eta
          - 10.0L * sigma;
    ph[5] = pi * (38645.0L / 756.0L - 65.0L / 9.0L * eta) * (1.0L + 3.0L * logl(v / vlso));
    ph[6] = 11583231236531.0L / 4694215680.0L - 640.0L / 3.0L * pi2
          - 6848.0L / 21.0L * OR_EULER_GAMMA - 6848.0L / 21.0L * logl(4.0L * v)
          + (-15737765635.0L / 3048192.0L + 2255.0L / 12.0L * pi2) * eta
          + 76055.0L / 1728.0L * eta * eta - 127825.0L / 1296.0L * eta * eta * eta;
    ph[7] = pi * (77096675.0L / 254016.0L + 378515.0L / 1512.0L * eta
                  - 74045.0L / 756.0L * eta * eta);
    ld sum = 0;
    for (int k = 0; k < 8; k++) sum += ph[k] * powl(v, (ld)k);
    ld tid = -39.0L / 2.0L * LT * powl(v, 10.0L)
           + (-3115.0L / 64.0L * LT + 6595.0L / 364.0L * d * dLT) * powl(v, 12.0L);
    return 3.0L / (128.0L * eta * powl(v, 5.0L)) * (sum + tid);
}

/* tau*(f): Buonanno et al. 2009 Eq. (3.8b) (non-spinning, as the paper cites) */
static ld tau_star_l(ld Mc_s, ld eta, ld f)
{
    const ld pi = OR_PI, pi2 = OR_PI * OR_PI;
    ld M = Mc_s * powl(eta, -0.6L);
    ld v = cbrtl(pi * M * f);
    ld v2 = v * v;
    ld t = 1.0L
         + (743.0L / 252.0L + 11.0L / 3.0L * eta) * v2
         - 32.0L / 5.0L * pi * powl(v, 3.0L)
         + (3058673.0L / 508032.0L + 5429.0L / 504.0L * eta + 617.0L / 72.0L * eta * eta) * powl(v, 4.0L)
         + (-7729.0L / 252.0L + 13.0L / 3.0L * eta) * pi * powl(v, 5.0L)
         + (-10052469856691.0L / 23471078400.0L + 128.0L / 3.0L * pi2 + 6848.0L / 105.0L * OR_EULER_GAMMA
            + (3147553127.0L / 3048192.0L - 451.0L / 12.0L * pi2) * eta
            - 15211.0L / 1728.0L * eta * eta + 25565.0L / 1296.0L * eta * eta * eta
            + 3424.0L / 105.0L * logl(16.0L * v2)) * powl(v, 6.0L)
         + (-15419335.0L / 127008.0L - 75703.0L / 756.0L * eta + 14809.0L / 378.0L * eta * eta)
           * pi * powl(v, 7.0L);
    return 5.0L * M / (256.0L * eta * powl(v, 8.0L)) * t;
}

/* pattern functions by tensor contraction; L = local sidereal angle of the site */
static void antenna_l(ld lat, ld L, ld gam, ld zeta, ld theta, ld phi, ld psi,
                      ld *Fp, ld *Fx)
{
    ld eE[3] = { -sinl(L), cosl(L), 0.0L };
    ld eN[3] = { -sinl(lat) * cosl(L), -sinl(lat) * sinl(L), cosl(lat) };
    ld u[3], w[3], D[3][3];
    ld au = gam - zeta / 2, aw = gam + zeta / 2;
    for (int i = 0; i < 3; i++) {
        u[i] = cosl(au) * eE[i] + sinl(au) * eN[i];
        w[i] = cosl(aw) * eE[i] + sinl(aw) * eN[i];
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D[i][j] = 0.5L * (u[i] * u[j] - w[i] * w[j]);
    ld eth[3] = { cosl(theta) * cosl(phi), cosl(theta) * sinl(phi), -sinl(theta) };
    ld eph[3] = { -sinl(phi), cosl(phi), 0.0L };
    ld p[3], q[3];
    for (int i = 0; i < 3; i++) {
        p[i] = cosl(psi) * eph[i] + sinl(psi) * eth[i];
        q[i] = -sinl(psi) * eph[i] + cosl(psi) * eth[i];
    }
    ld sp = 0, sx = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            sp += D[i][j] * (p[i] * p[j] - q[i] * q[j]);
            sx += D[i][j] * (p[i] * q[j] + q[i] * p[j]);
        }
    *Fp = sp; *Fx = sx;
}

/* strain of one arm on n frequencies; th = full parameter vector (Msun, Gpc, s, rad) */
static void strain_arm(const ld *th, const arm_t *a, int rotation, ld tc_fid,
                       int n, const ld *f, cld *h)
{
    ld Mc_s = th[I_MC] * OR_TSUN;
    ld dL_s = th[I_DL] * 1.0e3L * OR_MPC / OR_C;
    ld ci = cosl(th[I_IOTA]);
    ld cp = 0.5L * (1.0L + ci * ci);
    ld nh[3] = { sinl(th[I_TH]) * cosl(th[I_PH]), sinl(th[I_TH]) * sinl(th[I_PH]), cosl(th[I_TH]) };
    ld OmE = 2.0L * OR_PI / OR_TSID;
    for (int k = 0; k < n; k++) {
        ld fk = f[k];
        ld A = sqrtl(5.0L / 24.0L) * powl(OR_PI, -2.0L / 3.0L) * powl(Mc_s, 5.0L / 6.0L)
             * powl(fk, -7.0L / 6.0L) / dL_s;
        ld tau = tau_star_l(Mc_s, th[I_ETA], fk);
        ld gE = rotation ? OmE * (th[I_TC] - tau) : OmE * tc_fid;
        ld L = a->lon + gE;
        ld Fp, Fx;
        antenna_l(a->lat, L, a->gam, a->zeta, th[I_TH], th[I_PH], th[I_PSI], &Fp, &Fx);
        ld rh[3] = { cosl(a->lat) * cosl(L), cosl(a->lat) * sinl(L), sinl(a->lat) };
        ld PhiD = 2.0L * OR_PI * fk * (OR_REARTH / OR_C) * (rh[0] * nh[0] + rh[1] * nh[1] + rh[2] * nh[2]);
        ld Psi = psi_pn_l(Mc_s, th[I_ETA], th[I_CHI1], th[I_CHI2], th[I_LT], th[I_DLT], fk);
        ld Phi = 2.0L * OR_PI * fk * (th[I_TC] - tc_fid) - th[I_PHIC] - OR_PI / 4.0L + Psi + PhiD;
        cld Q = A * (Fp * cp + I * Fx * ci);
        h[k] = Q * (cosl(Phi) + I * sinl(Phi));
    }
}

/* the literal log grid and trapezoid weights */
static void make_grid(ld fmin, ld fmax, int n, ld *f, ld *w)
{
    for (int k = 0; k < n; k++)
        f[k] = (n == 1) ? fmin : fmin * powl(fmax / fmin, (ld)k / (ld)(n - 1));
    for (int k = 0; k < n; k++) {
        ld lo = (k > 0) ? f[k] - f[k - 1] : 0.0L;
        ld hi = (k < n - 1) ? f[k + 1] - f[k] : 0.0L;
        w[k] = 0.5L * (lo + hi);
    }
}

/* Fisher parameter slots per parameter set */
static int fisher_slots(int pset, int *slot)
{
    int base[9] = { I_MC, I_ETA, I_DL, I_TH, I_PH, I_IOTA, I_PSI, I_TC, I_PHIC };
    for (int i = 0; i < 9; i++) slot[i] = base[i];
    if (pset == 0) return 9;
    if (pset == 1) { slot[9] = I_CHI1; slot[10] = I_CHI2; return 11; }
    slot[9] = I_LT; slot[10] = I_DLT; return 11;
}

static void load_event(const double *ev, ld *th)
{
    for (int i = 0; i < N_ALL; i++) th[i] = ev[i];
}

static int check_event(const ld *th, ld fmin, ld fmax, int n)
{
    int st = 0;
    if (!(th[I_MC] > 0) || !(th[I_ETA] > 0) || !(th[I_ETA] <= 0.25L) || !(th[I_DL] > 0)) st |= ST_BAD_PARAM;
    if (!(fmax > fmin) || n < 2 || !(fmin > 0)) st |= ST_EMPTY_GRID;
    return st;
}

/* ------------------------------------------------------------------ */
/* exported: catalog preparation (Sec. 2.1)                            */
/*  in : m1, m2 [Msun], chi1z, chi2z, Lam1, Lam2 (may be NULL), dL_Mpc,
 *       redshift flag per event (1: masses are source-frame, apply (1+z),
 *       z = H0 dL / c), tcoal [sidereal days]
 *  out: Mc [Msun], eta, dL [Gpc], chi1z, chi2z (after m1>=m2 swap),
 *       LamT, dLamT, tc [s], fisco [Hz]                                  */
int or_prepare(int64_t n, const double *m1, const double *m2, const double *chi1,
               const double *chi2, const double *lam1, const double *lam2,
               const double *dL_Mpc, const uint8_t *zflag, const double *tcoal,
               double *Mc, double *eta, double *dL_Gpc, double *chi1o, double *chi2o,
               double *LamT, double *dLamT, double *tc_s, double *fisco)
{
    for (int64_t e = 0; e < n; e++) {
        ld a = m1[e], b = m2[e], ca = chi1[e], cb = chi2[e];
        ld la = lam1 ? lam1[e] : 0.0L, lb = lam2 ? lam2[e] : 0.0L;
        if (b > a) { ld t = a; a = b; b = t; t = ca; ca = cb; cb = t; t = la; la = lb; lb = t; }
        ld z = zflag[e] ? OR_H0 * (ld)dL_Mpc[e] / OR_CKMS : 0.0L;
        a *= (1.0L + z); b *= (1.0L + z);
        ld M = a + b;
        ld et = a * b / (M * M);
        ld mc = M * powl(et, 0.6L);
        ld d = (a - b) / M;   /* sqrt(1 - 4 eta) for m1 >= m2 */
        ld lt = 8.0L / 13.0L * ((1.0L + 7.0L * et - 31.0L * et * et) * (la + lb)
                + d * (1.0L + 9.0L * et - 11.0L * et * et) * (la - lb));
        ld dlt = 0.5L * (d * (1.0L - 13272.0L / 1319.0L * et + 8944.0L / 1319.0L * et * et) * (la + lb)
                 + (1.0L - 15910.0L / 1319.0L * et + 32850.0L / 1319.0L * et * et
                    + 3380.0L / 1319.0L * et * et * et) * (la - lb));
        Mc[e] = (double)mc; eta[e] = (double)et; dL_Gpc[e] = (double)((ld)dL_Mpc[e] / 1.0e3L);
        chi1o[e] = (double)ca; chi2o[e] = (double)cb;
        LamT[e] = (double)lt; dLamT[e] = (double)dlt;
        tc_s[e] = (double)((ld)tcoal[e] * OR_TSID);
        fisco[e] = (double)(1.0L / (powl(6.0L, 1.5L) * OR_PI * M * OR_TSUN));
    }
    return 0;
}

/* exported scalar pieces (for pins) */
double or_psi_pn(double Mc, double eta, double chi1, double chi2, double LT, double dLT, double f)
{
    return (double)psi_pn_l((ld)Mc * OR_TSUN, eta, chi1, chi2, LT, dLT, f);
}
double or_tau_star(double Mc, double eta, double f)
{
    return (double)tau_star_l((ld)Mc * OR_TSUN, eta, f);
}
void or_antenna(double lat, double L, double gam, double zeta, double theta, double phi,
                double psi, double *Fp, double *Fx)
{
    ld a, b;
    antenna_l(lat, L, gam, zeta, theta, phi, psi, &a, &b);
    *Fp = (double)a; *Fx = (double)b;
}

/* strain of every arm of the network on the event grid.
 * ev = 13 doubles (full parameter vector), out re/im = [n_arms][npts]        */
int or_strain(const double *ev, double fmin, double fmax, int npts, int ndet,
              const double *det, int rotation, double *f_out, double *re, double *im)
{
    arm_t arms[64];
    int na = expand_arms(ndet, det, arms, 64);
    if (na < 0) return -1;
    ld th[N_ALL]; load_event(ev, th);
    ld *f = malloc(sizeof(ld) * npts), *w = malloc(sizeof(ld) * npts);
    cld *h = malloc(sizeof(cld) * npts);
    make_grid(fmin, fmax, npts, f, w);
    for (int k = 0; k < npts; k++) f_out[k] = (double)f[k];
    for (int a = 0; a < na; a++) {
        strain_arm(th, &arms[a], rotation, th[I_TC], npts, f, h);
        for (int k = 0; k < npts; k++) {
            re[(size_t)a * npts + k] = (double)creall(h[k]);
            im[(size_t)a * npts + k] = (double)cimagl(h[k]);
        }
    }
    free(f); free(w); free(h);
    return na;
}

/* ------------------------------------------------------------------ */
/* SNR (Sec. 3.2): per event network SNR and optional per-arm SNR        */
static ld snr2_event(const ld *th, ld tc_fid, ld fmin, ld fmax, int npts, int na,
                     const arm_t *arms, const double *psd, int rotation, ld *per_arm)
{
    ld *f = malloc(sizeof(ld) * npts), *w = malloc(sizeof(ld) * npts);
    cld *h = malloc(sizeof(cld) * npts);
    make_grid(fmin, fmax, npts, f, w);
    ld tot = 0;
    for (int a = 0; a < na; a++) {
        strain_arm(th, &arms[a], rotation, tc_fid, npts, f, h);
        ld s = 0;
        for (int k = 0; k < npts; k++) {
            ld m2 = creall(h[k]) * creall(h[k]) + cimagl(h[k]) * cimagl(h[k]);
            s += 4.0L * w[k] * m2 / psd_eval(psd, arms[a].psd, f[k]);
        }
        if (per_arm) per_arm[a] = s;
        tot += s;
    }
    free(f); free(w); free(h);
    return tot;
}

int or_snr(int64_t n, const double *ev, const double *fmin, const double *fmax,
           const int32_t *npts, const uint32_t *arm_mask, int ndet, const double *det,
           int npsd, const double *psd, int rotation, double *snr, double *snr_arm,
           int32_t *status)
{
    (void)npsd;
    arm_t all[64], arms[64];
    int na = expand_arms(ndet, det, all, 64);
    if (na < 0 || (arm_mask && na > 32)) return -1;
    ld per[64];
    for (int64_t e = 0; e < n; e++) {
        ld th[N_ALL]; load_event(ev + N_ALL * e, th);
        int st = check_event(th, fmin[e], fmax[e], npts[e]);
        status[e] = st;
        if (st) {
            snr[e] = NAN;
            if (snr_arm) for (int a = 0; a < na; a++) snr_arm[(size_t)e * na + a] = NAN;
            continue;
        }
        int non = select_arms(all, na, arm_mask, e, arms);
        ld s2 = snr2_event(th, th[I_TC], fmin[e], fmax[e], npts[e], non, arms, psd, rotation, per);
        snr[e] = (double)sqrtl(s2);
        if (snr_arm)
            for (int a = 0, b = 0; a < na; a++) {
                int on = !arm_mask || ((arm_mask[e] >> a) & 1u);
                snr_arm[(size_t)e * na + a] = on ? (double)sqrtl(per[b++]) : 0.0;
            }
    }
    return na;
}

/* ------------------------------------------------------------------ */
/* Richardson-extrapolated central differences of the strain            */
#define RICH_LEVELS 4

/* target phase excursion of the first Richardson step (radians); a knob for the
 * step-insensitivity test, 0.1 by default */
static ld g_fd_target = 0.1L;
void or_set_fd_target(double t) { g_fd_target = (t > 0) ? (ld)t : 0.1L; }

/* pilot estimate of max_k |d ln h / d theta_i| on the grid, all arms */
static ld pilot_rate(const ld *th, int slot, ld tc_fid, int npts, const ld *f, int na,
                     const arm_t *arms, int rotation, cld *hp, cld *hm, cld *h0)
{
    static const ld pstep[N_ALL] = { 0, 1e-8L, 0, 1e-7L, 1e-7L, 1e-7L, 1e-7L, 1e-6L, 1e-6L,
                                     1e-6L, 1e-6L, 1e-3L, 1e-3L };
    ld dp = pstep[slot];
    if (slot == I_MC) dp = 1e-7L * th[I_MC];
    if (slot == I_DL) dp = 1e-6L * th[I_DL];
    if (slot == I_ETA) dp = fminl(dp, 0.4L * (0.25L - th[I_ETA]));
    ld tp[N_ALL], tm[N_ALL];
    ld rate = 0;
    for (int a = 0; a < na; a++) {
        memcpy(tp, th, sizeof tp); memcpy(tm, th, sizeof tm);
        tp[slot] += dp; tm[slot] -= dp;
        strain_arm(th, &arms[a], rotation, tc_fid, npts, f, h0);
        strain_arm(tp, &arms[a], rotation, tc_fid, npts, f, hp);
        strain_arm(tm, &arms[a], rotation, tc_fid, npts, f, hm);
        ld hmax = 0;
        for (int k = 0; k < npts; k++) hmax = fmaxl(hmax, cabsl(h0[k]));
        for (int k = 0; k < npts; k++) {
            ld m = cabsl(h0[k]);
            if (m <= 1e-6L * hmax) continue;
            rate = fmaxl(rate, cabsl(hp[k] - hm[k]) / (2.0L * dp * m));
        }
    }
    return rate;
}

/* choose the first Richardson step of each Fisher parameter */
static void choose_steps(const ld *th, ld tc_fid, int P, const int *slot, int npts, const ld *f,
                         int na, const arm_t *arms, int rotation, ld *step)
{
    cld *hp = malloc(sizeof(cld) * npts), *hm = malloc(sizeof(cld) * npts),
        *h0 = malloc(sizeof(cld) * npts);
    for (int i = 0; i < P; i++) {
        int s = slot[i];
        ld r = pilot_rate(th, s, tc_fid, npts, f, na, arms, rotation, hp, hm, h0);
        ld d0 = (r > 0) ? g_fd_target / r : 1.0L;
        if (s == I_MC) d0 = fminl(d0, 0.05L * th[I_MC]);
        if (s == I_DL) d0 = fminl(d0, 0.05L * th[I_DL]);
        if (s == I_ETA) d0 = fminl(d0, 0.3L * fminl(th[I_ETA], 0.25L - th[I_ETA]));
        /* angles that move only the amplitude (iota near 0 or pi) have small
         * rates and would get steps near 1 rad: cap them so the Richardson
         * truncation error stays far below the derivative's size */
        if (s == I_TH || s == I_PH || s == I_IOTA || s == I_PSI || s == I_PHIC)
            d0 = fminl(d0, 0.05L);
        step[i] = d0;
    }
    free(hp); free(hm); free(h0);
}

/* derivative of one arm's strain w.r.t. slot s, at all grid points       */
static void fd_deriv_arm(const ld *th, int s, ld d0, ld tc_fid, int npts, const ld *f,
                         const arm_t *arm, int rotation, cld *out, ld *errbar,
                         cld *hp, cld *hm, cld **R)
{
    ld tp[N_ALL], tm[N_ALL];
    for (int m = 0; m < RICH_LEVELS; m++) {
        ld d = d0 / (ld)(1 << m);
        memcpy(tp, th, sizeof tp); memcpy(tm, th, sizeof tm);
        tp[s] += d; tm[s] -= d;
        strain_arm(tp, arm, rotation, tc_fid, npts, f, hp);
        strain_arm(tm, arm, rotation, tc_fid, npts, f, hm);
        /* divide by the step actually taken (the rounded tp - tm), not by 2d */
        ld span = tp[s] - tm[s];
        for (int k = 0; k < npts; k++) R[m][k] = (hp[k] - hm[k]) / span;
    }
    /* Neville table in d^2 with ratio 4 */
    for (int k = 0; k < npts; k++) {
        cld T[RICH_LEVELS][RICH_LEVELS];
        for (int m = 0; m < RICH_LEVELS; m++) T[m][0] = R[m][k];
        for (int j = 1; j < RICH_LEVELS; j++)
            for (int m = j; m < RICH_LEVELS; m++) {
                ld fac = powl(4.0L, (ld)j) - 1.0L;
                T[m][j] = T[m][j - 1] + (T[m][j - 1] - T[m - 1][j - 1]) / fac;
            }
        out[k] = T[RICH_LEVELS - 1][RICH_LEVELS - 1];
        if (errbar) errbar[k] = cabsl(T[RICH_LEVELS - 1][RICH_LEVELS - 1]
                                      - T[RICH_LEVELS - 2][RICH_LEVELS - 2]);
    }
}

/* Fisher of one event with given (or chosen) steps; returns 0 or status   */
static int fisher_event(const ld *th, ld tc_fid, ld fmin, ld fmax, int npts, int P, const int *slot,
                        int na, const arm_t *arms, const double *psd, int rotation,
                        const ld *steps_in, ld *steps_out, ld *G, ld *snr2, ld *relerr)
{
    ld *f = malloc(sizeof(ld) * npts), *w = malloc(sizeof(ld) * npts);
    cld *D = malloc(sizeof(cld) * (size_t)P * npts);
    cld *hp = malloc(sizeof(cld) * npts), *hm = malloc(sizeof(cld) * npts);
    cld *h0 = malloc(sizeof(cld) * npts);
    cld *Rb[RICH_LEVELS];
    for (int m = 0; m < RICH_LEVELS; m++) Rb[m] = malloc(sizeof(cld) * npts);
    ld *eb = malloc(sizeof(ld) * npts);
    make_grid(fmin, fmax, npts, f, w);
    ld steps[16];
    if (steps_in) for (int i = 0; i < P; i++) steps[i] = steps_in[i];
    else choose_steps(th, tc_fid, P, slot, npts, f, na, arms, rotation, steps);
    if (steps_out) for (int i = 0; i < P; i++) steps_out[i] = steps[i];
    for (int i = 0; i < P * P; i++) G[i] = 0;
    ld s2 = 0, worst = 0;
    for (int a = 0; a < na; a++) {
        for (int i = 0; i < P; i++) {
            fd_deriv_arm(th, slot[i], steps[i], tc_fid, npts, f, &arms[a], rotation,
                         D + (size_t)i * npts, eb, hp, hm, Rb);
            /* Richardson error bar relative to the peak of |d_i h| on the grid */
            ld dmax = 0, emax = 0;
            for (int k = 0; k < npts; k++) {
                dmax = fmaxl(dmax, cabsl(D[(size_t)i * npts + k]));
                emax = fmaxl(emax, eb[k]);
            }
            if (dmax > 0) worst = fmaxl(worst, emax / dmax);
        }
        strain_arm(th, &arms[a], rotation, tc_fid, npts, f, h0);
        for (int k = 0; k < npts; k++) {
            ld wk = 4.0L * w[k] / psd_eval(psd, arms[a].psd, f[k]);
            s2 += wk * (creall(h0[k]) * creall(h0[k]) + cimagl(h0[k]) * cimagl(h0[k]));
            for (int i = 0; i < P; i++) {
                cld di = D[(size_t)i * npts + k];
                for (int j = i; j < P; j++) {
                    cld dj = D[(size_t)j * npts + k];
                    G[i * P + j] += wk * creall(conjl(di) * dj);
                }
            }
        }
    }
    for (int i = 0; i < P; i++)
        for (int j = 0; j < i; j++) G[i * P + j] = G[j * P + i];
    *snr2 = s2;
    if (relerr) *relerr = worst;
    free(f); free(w); free(D); free(hp); free(hm); free(h0); free(eb);
    for (int m = 0; m < RICH_LEVELS; m++) free(Rb[m]);
    return 0;
}

/* exported Fisher: ev [n][13], pset [n]; out fisher [n][P][P] (full), snr [n],
 * fd_relerr [n] (largest Richardson error bar relative to |d_i h|, or NULL)   */
int or_fisher(int64_t n, const double *ev, const int8_t *pset, const double *fmin,
              const double *fmax, const int32_t *npts, const uint32_t *arm_mask, int ndet,
              const double *det, int npsd, const double *psd, int rotation, int n_par,
              double *fisher, double *snr, double *fd_relerr, int32_t *status)
{
    (void)npsd;
    arm_t all[64], arms[64];
    int na = expand_arms(ndet, det, all, 64);
    if (na < 0 || (arm_mask && na > 32)) return -1;
    ld G[16 * 16];
    for (int64_t e = 0; e < n; e++) {
        ld th[N_ALL]; load_event(ev + N_ALL * e, th);
        int slot[16];
        int P = fisher_slots(pset[e], slot);
        int st = check_event(th, fmin[e], fmax[e], npts[e]);
        if (P != n_par) st |= ST_BAD_PARAM;
        status[e] = st;
        double *Fo = fisher + (size_t)e * n_par * n_par;
        if (st) {
            for (int i = 0; i < n_par * n_par; i++) Fo[i] = NAN;
            snr[e] = NAN;
            if (fd_relerr) fd_relerr[e] = NAN;
            continue;
        }
        ld s2 = 0, re = 0;
        int non = select_arms(all, na, arm_mask, e, arms);
        if (non > 0)
            fisher_event(th, th[I_TC], fmin[e], fmax[e], npts[e], P, slot, non, arms, psd,
                         rotation, NULL, NULL, G, &s2, &re);
        else   /* every arm off: no signal, no information */
            for (int i = 0; i < P * P; i++) G[i] = 0;
        for (int i = 0; i < P * P; i++) Fo[i] = (double)G[i];
        snr[e] = (double)sqrtl(s2);
        if (fd_relerr) fd_relerr[e] = (double)re;
    }
    return na;
}

/* ------------------------------------------------------------------ */
/* Inversion (Sec. 4.1)                                                 */
static void jacobi_eig(int P, ld *A, ld *ev)
{
    /* cyclic Jacobi on a symmetric P x P matrix (destroys A) */
    for (int sweep = 0; sweep < 100; sweep++) {
        ld off = 0;
        for (int i = 0; i < P; i++)
            for (int j = i + 1; j < P; j++) off += A[i * P + j] * A[i * P + j];
        if (off < 1e-60L) break;
        for (int p = 0; p < P; p++)
            for (int q = p + 1; q < P; q++) {
                ld apq = A[p * P + q];
                if (fabsl(apq) < 1e-300L) continue;
                ld app = A[p * P + p], aqq = A[q * P + q];
                ld tau = (aqq - app) / (2.0L * apq);
                ld t = (tau >= 0 ? 1.0L : -1.0L) / (fabsl(tau) + sqrtl(1.0L + tau * tau));
                ld c = 1.0L / sqrtl(1.0L + t * t), s = t * c;
                for (int k = 0; k < P; k++) {
                    ld akp = A[k * P + p], akq = A[k * P + q];
                    A[k * P + p] = c * akp - s * akq;
                    A[k * P + q] = s * akp + c * akq;
                }
                for (int k = 0; k < P; k++) {
                    ld apk = A[p * P + k], aqk = A[q * P + k];
                    A[p * P + k] = c * apk - s * aqk;
                    A[q * P + k] = s * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < P; i++) ev[i] = A[i * P + i];
}

/* in: fisher [n][P][P]; out: cov [n][P][P], cond2 [n], inv_err [n], status [n] */
int or_invert(int64_t n, int P, const double *fisher, double cond_max, double *cov,
              double *cond2, double *inv_err, int32_t *status)
{
    for (int64_t e = 0; e < n; e++) {
        const double *G = fisher + (size_t)e * P * P;
        double *C = cov + (size_t)e * P * P;
        int st = 0;
        ld Gh[256], A[256], L[256], Li[256], Ch[256], d[16], ev[16];
        for (int i = 0; i < P * P; i++) if (!isfinite(G[i])) st |= ST_NONFINITE;
        for (int i = 0; i < P && !st; i++) {
            if (!(G[i * P + i] > 0)) st |= ST_NOT_PD;
            else d[i] = sqrtl((ld)G[i * P + i]);
        }
        if (st) {
            for (int i = 0; i < P * P; i++) C[i] = NAN;
            cond2[e] = NAN; inv_err[e] = NAN; status[e] = st;
            continue;
        }
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) Gh[i * P + j] = (ld)G[i * P + j] / (d[i] * d[j]);
        memcpy(A, Gh, sizeof(ld) * P * P);
        jacobi_eig(P, A, ev);
        ld emax = 0, emin = INFINITY;
        for (int i = 0; i < P; i++) { emax = fmaxl(emax, fabsl(ev[i])); emin = fminl(emin, fabsl(ev[i])); }
        ld kappa = (emin > 0) ? emax / emin : INFINITY;
        cond2[e] = (double)kappa;
        if (kappa > 1.0L / DBL_EPSILON) st |= ST_ILL_COND;
        if (kappa > cond_max) {
            st |= ST_COND_GT_MAX;
            for (int i = 0; i < P * P; i++) C[i] = NAN;
            inv_err[e] = NAN; status[e] = st;
            continue;
        }
        /* Cholesky Gh = L L^T */
        memset(L, 0, sizeof(ld) * P * P);
        for (int j = 0; j < P && !(st & ST_NOT_PD); j++) {
            ld s = Gh[j * P + j];
            for (int k = 0; k < j; k++) s -= L[j * P + k] * L[j * P + k];
            if (!(s > 0)) { st |= ST_NOT_PD; break; }
            L[j * P + j] = sqrtl(s);
            for (int i = j + 1; i < P; i++) {
                ld t = Gh[i * P + j];
                for (int k = 0; k < j; k++) t -= L[i * P + k] * L[j * P + k];
                L[i * P + j] = t / L[j * P + j];
            }
        }
        if (st & ST_NOT_PD) {
            for (int i = 0; i < P * P; i++) C[i] = NAN;
            inv_err[e] = NAN; status[e] = st;
            continue;
        }
        /* Li = L^{-1} by forward substitution on the identity */
        memset(Li, 0, sizeof(ld) * P * P);
        for (int c = 0; c < P; c++)
            for (int i = c; i < P; i++) {
                ld s = (i == c) ? 1.0L : 0.0L;
                for (int k = c; k < i; k++) s -= L[i * P + k] * Li[k * P + c];
                Li[i * P + c] = s / L[i * P + i];
            }
        /* Ch = Li^T Li */
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) {
                ld s = 0;
                for (int k = 0; k < P; k++) s += Li[k * P + i] * Li[k * P + j];
                Ch[i * P + j] = s;
            }
        ld Cl[256];
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) {
                Cl[i * P + j] = Ch[i * P + j] / (d[i] * d[j]);
                C[i * P + j] = (double)Cl[i * P + j];
            }
        ld eps = 0;
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) {
                ld s = 0;
                for (int k = 0; k < P; k++) s += (ld)G[i * P + k] * (ld)C[k * P + j];
                eps = fmaxl(eps, fabsl(s - (i == j ? 1.0L : 0.0L)));
            }
        inv_err[e] = (double)eps;
        status[e] = st;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Covariance tools (Sec. 4.1 and the manipulations listed in Sec. 4.2)  */

/* cyclic Jacobi with eigenvectors: A = V diag(w) V^T (A destroyed; V[i*P+k] =
 * component i of eigenvector k); eigenpairs sorted by increasing w and each
 * eigenvector's largest-magnitude component made positive              */
static void jacobi_eigv(int P, ld *A, ld *w, ld *V)
{
    for (int i = 0; i < P * P; i++) V[i] = 0;
    for (int i = 0; i < P; i++) V[i * P + i] = 1;
    for (int sweep = 0; sweep < 100; sweep++) {
        ld off = 0, tot = 0;
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) {
                tot += A[i * P + j] * A[i * P + j];
                if (i != j) off += A[i * P + j] * A[i * P + j];
            }
        if (off <= 1e-64L * tot) break;
        for (int p = 0; p < P; p++)
            for (int q = p + 1; q < P; q++) {
                ld apq = A[p * P + q];
                if (apq == 0) continue;
                ld tau = (A[q * P + q] - A[p * P + p]) / (2.0L * apq);
                ld t = (tau >= 0 ? 1.0L : -1.0L) / (fabsl(tau) + sqrtl(1.0L + tau * tau));
                ld c = 1.0L / sqrtl(1.0L + t * t), sn = t * c;
                for (int k = 0; k < P; k++) {
                    ld akp = A[k * P + p], akq = A[k * P + q];
                    A[k * P + p] = c * akp - sn * akq;
                    A[k * P + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < P; k++) {
                    ld apk = A[p * P + k], aqk = A[q * P + k];
                    A[p * P + k] = c * apk - sn * aqk;
                    A[q * P + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < P; k++) {
                    ld vkp = V[k * P + p], vkq = V[k * P + q];
                    V[k * P + p] = c * vkp - sn * vkq;
                    V[k * P + q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < P; i++) w[i] = A[i * P + i];
    for (int a = 0; a < P; a++) {              /* selection sort, ascending */
        int m = a;
        for (int b = a + 1; b < P; b++) if (w[b] < w[m]) m = b;
        if (m != a) {
            ld t = w[a]; w[a] = w[m]; w[m] = t;
            for (int i = 0; i < P; i++) { t = V[i * P + a]; V[i * P + a] = V[i * P + m]; V[i * P + m] = t; }
        }
    }
    for (int k = 0; k < P; k++) {
        int im = 0;
        for (int i = 1; i < P; i++) if (fabsl(V[i * P + k]) > fabsl(V[im * P + k])) im = i;
        if (V[im * P + k] < 0) for (int i = 0; i < P; i++) V[i * P + k] = -V[i * P + k];
    }
}

/* Eigenvalues (ascending) and eigenvectors of each Fisher matrix, optionally
 * of the matrix normalised by sqrt(diag) (CheckFisher, Sec. 4.1).
 * in: fisher [n][P][P]; out: w [n][P], V [n][P][P] (V[e][i][k] = component i
 * of eigenvector k), either may be NULL.                                 */
int or_fisher_eig(int64_t n, int P, const double *fisher, int normalize, double *w, double *V)
{
    for (int64_t e = 0; e < n; e++) {
        const double *G = fisher + (size_t)e * P * P;
        ld A[256], wl[16], Vl[256], d[16];
        int norm = normalize;
        for (int i = 0; i < P; i++) if (!(G[i * P + i] > 0)) norm = 0;
        for (int i = 0; i < P; i++) d[i] = norm ? sqrtl((ld)G[i * P + i]) : 1.0L;
        for (int i = 0; i < P; i++)
            for (int j = 0; j < P; j++) A[i * P + j] = (ld)G[i * P + j] / (d[i] * d[j]);
        jacobi_eigv(P, A, wl, Vl);
        if (w) for (int i = 0; i < P; i++) w[(size_t)e * P + i] = (double)wl[i];
        if (V) for (int i = 0; i < P * P; i++) V[(size_t)e * P * P + i] = (double)Vl[i];
    }
    return 0;
}

/* Covariance with the options of CovMatr and the Fisher manipulations of
 * Sec. 4.1-4.2.  For every event:
 *   1. fixParams: keep only the parameters whose bit is set in `keep`
 *      (rows and columns of fixed parameters removed before inversion);
 *   2. addPrior: add prior[i] (if prior != NULL, indexed by the original
 *      parameter slot) to the diagonal of the kept matrix;
 *   3. normalise rows and columns by sqrt(diag) unless a diagonal element is
 *      not positive (then no normalisation);
 *   4. condition number = ratio of the largest to the smallest |eigenvalue|
 *      of the normalised matrix; above cond_max the matrix is not inverted;
 *   5. invert by `method`: 0 Cholesky; 1 Cholesky, SVD when not positive
 *      definite (status bit 128); 2 SVD; 3 SVD with singular values below
 *      thresh * max replaced by thresh * max; 4 SVD with them left out;
 *      5 LU with partial pivoting.  The SVD of the symmetric matrix is its
 *      eigendecomposition (singular values |w|, the signs kept on one side);
 *   6. undo the normalisation; eps = max |Gamma C - 1| with the kept, prior-
 *      added Gamma and the double-rounded C.
 * out: cov [n][Pk][Pk] (Pk = number of kept parameters), cond2, inv_err, status */
int or_covariance(int64_t n, int P, const double *fisher, uint32_t keep, const double *prior,
                  int method, double thresh, double cond_max, double *cov, double *cond2,
                  double *inv_err, int32_t *status)
{
    int idx[16], Pk = 0;
    for (int i = 0; i < P; i++) if ((keep >> i) & 1u) idx[Pk++] = i;
    if (Pk == 0) return -1;
    for (int64_t e = 0; e < n; e++) {
        const double *Gf = fisher + (size_t)e * P * P;
        double *C = cov + (size_t)e * Pk * Pk;
        ld G[256], Gh[256], A[256], Ch[256], d[16], w[16], V[256];
        int st = 0;
        for (int a = 0; a < Pk; a++)
            for (int b = 0; b < Pk; b++) {
                G[a * Pk + b] = (ld)Gf[idx[a] * P + idx[b]];
                if (a == b && prior) G[a * Pk + b] += (ld)prior[idx[a]];
                if (!isfinite((double)G[a * Pk + b])) st |= ST_NONFINITE;
            }
        if (st) {
            for (int i = 0; i < Pk * Pk; i++) C[i] = NAN;
            cond2[e] = NAN; inv_err[e] = NAN; status[e] = st;
            continue;
        }
        int norm = 1;
        for (int a = 0; a < Pk; a++) if (!(G[a * Pk + a] > 0)) norm = 0;
        for (int a = 0; a < Pk; a++) d[a] = norm ? sqrtl(G[a * Pk + a]) : 1.0L;
        for (int a = 0; a < Pk; a++)
            for (int b = 0; b < Pk; b++) Gh[a * Pk + b] = G[a * Pk + b] / (d[a] * d[b]);
        memcpy(A, Gh, sizeof(ld) * Pk * Pk);
        jacobi_eigv(Pk, A, w, V);
        ld smax = 0, smin = INFINITY;
        for (int a = 0; a < Pk; a++) { smax = fmaxl(smax, fabsl(w[a])); smin = fminl(smin, fabsl(w[a])); }
        ld kappa = smin > 0 ? smax / smin : INFINITY;
        cond2[e] = (double)kappa;
        if (kappa > 1.0L / DBL_EPSILON) st |= ST_ILL_COND;
        if (kappa > cond_max) {
            st |= ST_COND_GT_MAX;
            for (int i = 0; i < Pk * Pk; i++) C[i] = NAN;
            inv_err[e] = NAN; status[e] = st;
            continue;
        }
        int use_svd = method >= 2 && method <= 4;
        if (method == 0 || method == 1) {
            /* Cholesky Gh = L L^T, C = L^-T L^-1 */
            ld L[256], Li[256];
            memset(L, 0, sizeof L);
            int pd = 1;
            for (int j = 0; j < Pk && pd; j++) {
                ld sj = Gh[j * Pk + j];
                for (int k = 0; k < j; k++) sj -= L[j * Pk + k] * L[j * Pk + k];
                if (!(sj > 0)) { pd = 0; break; }
                L[j * Pk + j] = sqrtl(sj);
                for (int i = j + 1; i < Pk; i++) {
                    ld t = Gh[i * Pk + j];
                    for (int k = 0; k < j; k++) t -= L[i * Pk + k] * L[j * Pk + k];
                    L[i * Pk + j] = t / L[j * Pk + j];
                }
            }
            if (!pd) {
                st |= ST_NOT_PD;
                if (method == 0) {
                    for (int i = 0; i < Pk * Pk; i++) C[i] = NAN;
                    inv_err[e] = NAN; status[e] = st;
                    continue;
                }
                st |= ST_SVD_FALLBACK;
                use_svd = 1;
            } else {
                memset(Li, 0, sizeof Li);
                for (int c = 0; c < Pk; c++)
                    for (int i = c; i < Pk; i++) {
                        ld t = (i == c) ? 1.0L : 0.0L;
                        for (int k = c; k < i; k++) t -= L[i * Pk + k] * Li[k * Pk + c];
                        Li[i * Pk + c] = t / L[i * Pk + i];
                    }
                for (int i = 0; i < Pk; i++)
                    for (int j = 0; j < Pk; j++) {
                        ld t = 0;
                        for (int k = 0; k < Pk; k++) t += Li[k * Pk + i] * Li[k * Pk + j];
                        Ch[i * Pk + j] = t;
                    }
            }
        }
        if (use_svd) {
            /* inverse singular values: 1/w, with the small ones (|w| < thresh smax)
             * replaced (method 3) or dropped (method 4) */
            ld iw[16];
            for (int k = 0; k < Pk; k++) {
                ld a = fabsl(w[k]);
                if (method == 3 && a < (ld)thresh * smax)
                    iw[k] = (w[k] < 0 ? -1.0L : 1.0L) / ((ld)thresh * smax);
                else if (method == 4 && a < (ld)thresh * smax)
                    iw[k] = 0;
                else
                    iw[k] = 1.0L / w[k];
            }
            for (int i = 0; i < Pk; i++)
                for (int j = 0; j < Pk; j++) {
                    ld t = 0;
                    for (int k = 0; k < Pk; k++) t += V[i * Pk + k] * iw[k] * V[j * Pk + k];
                    Ch[i * Pk + j] = t;
                }
        } else if (method == 5) {
            /* LU with partial pivoting, P Gh = L U, then columns of the inverse */
            ld LU[256];
            int piv[16];
            memcpy(LU, Gh, sizeof(ld) * Pk * Pk);
            for (int i = 0; i < Pk; i++) piv[i] = i;
            int sing = 0;
            for (int k = 0; k < Pk; k++) {
                int m = k;
                for (int i = k + 1; i < Pk; i++) if (fabsl(LU[i * Pk + k]) > fabsl(LU[m * Pk + k])) m = i;
                if (LU[m * Pk + k] == 0) { sing = 1; break; }
                if (m != k) {
                    for (int j = 0; j < Pk; j++) { ld t = LU[k * Pk + j]; LU[k * Pk + j] = LU[m * Pk + j]; LU[m * Pk + j] = t; }
                    int t = piv[k]; piv[k] = piv[m]; piv[m] = t;
                }
                for (int i = k + 1; i < Pk; i++) {
                    LU[i * Pk + k] /= LU[k * Pk + k];
                    for (int j = k + 1; j < Pk; j++) LU[i * Pk + j] -= LU[i * Pk + k] * LU[k * Pk + j];
                }
            }
            if (sing) {
                st |= ST_NOT_PD;
                for (int i = 0; i < Pk * Pk; i++) C[i] = NAN;
                inv_err[e] = NAN; status[e] = st;
                continue;
            }
            for (int c = 0; c < Pk; c++) {
                ld y[16];
                for (int i = 0; i < Pk; i++) {
                    ld t = (piv[i] == c) ? 1.0L : 0.0L;
                    for (int k = 0; k < i; k++) t -= LU[i * Pk + k] * y[k];
                    y[i] = t;
                }
                for (int i = Pk - 1; i >= 0; i--) {
                    ld t = y[i];
                    for (int k = i + 1; k < Pk; k++) t -= LU[i * Pk + k] * Ch[k * Pk + c];
                    Ch[i * Pk + c] = t / LU[i * Pk + i];
                }
            }
        }
        for (int a = 0; a < Pk; a++)
            for (int b = 0; b < Pk; b++) C[a * Pk + b] = (double)(Ch[a * Pk + b] / (d[a] * d[b]));
        ld eps = 0;
        for (int a = 0; a < Pk; a++)
            for (int b = 0; b < Pk; b++) {
                ld t = 0;
                for (int k = 0; k < Pk; k++) t += G[a * Pk + k] * (ld)C[k * Pk + b];
                eps = fmaxl(eps, fabsl(t - (a == b ? 1.0L : 0.0L)));
            }
        inv_err[e] = (double)eps;
        status[e] = st;
    }
    return Pk;
}

/* Sky-localisation area at confidence level perc (percent), Sec. 4.1:
 * Delta Omega = -2 pi |sin theta| sqrt(C_tt C_pp - C_tp^2) ln(1 - perc/100),
 * in steradians (units 0) or square degrees (units 1).
 * in: cov [n][P][P], theta [n]; slots it, ip of theta and phi; out: area [n] */
int or_sky_area(int64_t n, int P, const double *cov, int it, int ip, const double *theta,
                double perc, int units, double *area)
{
    for (int64_t e = 0; e < n; e++) {
        const double *C = cov + (size_t)e * P * P;
        ld det = (ld)C[it * P + it] * (ld)C[ip * P + ip] - (ld)C[it * P + ip] * (ld)C[it * P + ip];
        ld a = -2.0L * OR_PI * fabsl(sinl((ld)theta[e])) * sqrtl(det) * log1pl(-(ld)perc / 100.0L);
        if (units == 1) a *= (180.0L / OR_PI) * (180.0L / OR_PI);
        area[e] = (double)a;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* VJP references by Richardson differences                             */

/* d SNR / d theta_i for the event's Fisher parameters; out grad [n][P]  */
int or_snr_grad(int64_t n, const double *ev, const int8_t *pset, const double *fmin,
                const double *fmax, const int32_t *npts, const uint32_t *arm_mask, int ndet,
                const double *det, int npsd, const double *psd, int rotation, int n_par,
                double *grad)
{
    (void)npsd;
    arm_t all[64], arms[64];
    int na = expand_arms(ndet, det, all, 64);
    if (na < 0 || (arm_mask && na > 32)) return -1;
    for (int64_t e = 0; e < n; e++) {
        ld th[N_ALL]; load_event(ev + N_ALL * e, th);
        int slot[16];
        int P = fisher_slots(pset[e], slot);
        double *g = grad + (size_t)e * n_par;
        if (P != n_par || check_event(th, fmin[e], fmax[e], npts[e])) {
            for (int i = 0; i < n_par; i++) g[i] = NAN;
            continue;
        }
        ld tc_fid = th[I_TC];
        int non = select_arms(all, na, arm_mask, e, arms);
        for (int i = 0; i < P; i++) {
            int s = slot[i];
            ld d0;
            switch (s) {
            case I_MC: d0 = 1e-3L * th[I_MC]; break;
            case I_ETA: d0 = fminl(1e-3L, 0.3L * fminl(th[I_ETA], 0.25L - th[I_ETA])); break;
            case I_DL: d0 = 1e-2L * th[I_DL]; break;
            case I_TC: d0 = 50.0L; break;
            case I_LT: case I_DLT: d0 = 5.0L; break;
            default: d0 = 1e-2L;
            }
            ld R[RICH_LEVELS][RICH_LEVELS];
            for (int m = 0; m < RICH_LEVELS; m++) {
                ld d = d0 / (ld)(1 << m);
                ld tp[N_ALL], tm[N_ALL];
                memcpy(tp, th, sizeof tp); memcpy(tm, th, sizeof tm);
                tp[s] += d; tm[s] -= d;
                ld sp = sqrtl(snr2_event(tp, tc_fid, fmin[e], fmax[e], npts[e], non, arms, psd, rotation, NULL));
                ld sm = sqrtl(snr2_event(tm, tc_fid, fmin[e], fmax[e], npts[e], non, arms, psd, rotation, NULL));
                R[m][0] = (sp - sm) / (tp[s] - tm[s]);
            }
            for (int j = 1; j < RICH_LEVELS; j++)
                for (int m = j; m < RICH_LEVELS; m++)
                    R[m][j] = R[m][j - 1] + (R[m][j - 1] - R[m - 1][j - 1]) / (powl(4.0L, (ld)j) - 1.0L);
            g[i] = (double)R[RICH_LEVELS - 1][RICH_LEVELS - 1];
        }
    }
    return na;
}

/* log det of a P x P symmetric positive matrix via Cholesky of the
 * normalised matrix; returns NAN if not positive definite               */
static ld logdet_l(int P, const ld *G)
{
    ld d[16], Gh[256], L[256];
    ld ld_sum = 0;
    for (int i = 0; i < P; i++) {
        if (!(G[i * P + i] > 0)) return NAN;
        d[i] = sqrtl(G[i * P + i]);
        ld_sum += 2.0L * logl(d[i]);
    }
    for (int i = 0; i < P; i++)
        for (int j = 0; j < P; j++) Gh[i * P + j] = G[i * P + j] / (d[i] * d[j]);
    memset(L, 0, sizeof(ld) * P * P);
    for (int j = 0; j < P; j++) {
        ld s = Gh[j * P + j];
        for (int k = 0; k < j; k++) s -= L[j * P + k] * L[j * P + k];
        if (!(s > 0)) return NAN;
        L[j * P + j] = sqrtl(s);
        ld_sum += logl(s);
        for (int i = j + 1; i < P; i++) {
            ld t = Gh[i * P + j];
            for (int k = 0; k < j; k++) t -= L[i * P + k] * L[j * P + k];
            L[i * P + j] = t / L[j * P + j];
        }
    }
    return ld_sum;
}

/* d (sum_e log det Gamma_e) / d gamma_d for the detectors listed in dets[]
 * (orientation of detector d, radians).  The Fisher derivative steps are
 * chosen once at the fiducial orientation and reused at every shifted one,
 * so the differenced quantity is one smooth function of gamma.
 * out: grad [n_d]; logdet [n] (fiducial, may be NULL)                     */
int or_logdet_grad_gamma(int64_t n, const double *ev, const int8_t *pset, const double *fmin,
                         const double *fmax, const int32_t *npts, const uint32_t *arm_mask,
                         int ndet, const double *det, int npsd, const double *psd, int rotation,
                         int n_par, int n_d, const int32_t *dets, double step0, double *grad,
                         double *logdet)
{
    (void)npsd;
    arm_t all[64], arms[64];
    int na = expand_arms(ndet, det, all, 64);
    if (na < 0 || (arm_mask && na > 32)) return -1;
    double *dcopy = malloc(sizeof(double) * 6 * ndet);
    ld G[256];
    for (int q = 0; q < n_d; q++) grad[q] = 0;
    for (int64_t e = 0; e < n; e++) {
        ld th[N_ALL]; load_event(ev + N_ALL * e, th);
        int slot[16];
        int P = fisher_slots(pset[e], slot);
        if (P != n_par || check_event(th, fmin[e], fmax[e], npts[e])) {
            for (int q = 0; q < n_d; q++) grad[q] = NAN;
            if (logdet) logdet[e] = NAN;
            continue;
        }
        ld steps[16], s2;
        int non = select_arms(all, na, arm_mask, e, arms);
        fisher_event(th, th[I_TC], fmin[e], fmax[e], npts[e], P, slot, non, arms, psd, rotation,
                     NULL, steps, G, &s2, NULL);
        if (logdet) logdet[e] = (double)logdet_l(P, G);
        for (int q = 0; q < n_d; q++) {
            ld R[RICH_LEVELS][RICH_LEVELS];
            for (int m = 0; m < RICH_LEVELS; m++) {
                ld d = (ld)step0 / (ld)(1 << m);
                ld vals[2], span_p = 0, span_m = 0;
                for (int sgn = 0; sgn < 2; sgn++) {
                    memcpy(dcopy, det, sizeof(double) * 6 * ndet);
                    arm_t a2[64], a2on[64];
                    expand_arms(ndet, dcopy, a2, 64);
                    /* shift the orientation of every arm of detector dets[q] */
                    int first = 0;
                    for (int dd = 0; dd < dets[q]; dd++) first += ((int)det[6 * dd + 4] == 0) ? 1 : 3;
                    int cnt = ((int)det[6 * dets[q] + 4] == 0) ? 1 : 3;
                    for (int a = first; a < first + cnt; a++) a2[a].gam += (sgn == 0 ? d : -d);
                    if (sgn == 0) span_p = a2[first].gam; else span_m = a2[first].gam;
                    int non2 = select_arms(a2, na, arm_mask, e, a2on);
                    fisher_event(th, th[I_TC], fmin[e], fmax[e], npts[e], P, slot, non2, a2on, psd,
                                 rotation, steps, NULL, G, &s2, NULL);
                    vals[sgn] = logdet_l(P, G);
                }
                R[m][0] = (vals[0] - vals[1]) / (span_p - span_m);
            }
            for (int j = 1; j < RICH_LEVELS; j++)
                for (int m = j; m < RICH_LEVELS; m++)
                    R[m][j] = R[m][j - 1] + (R[m][j - 1] - R[m - 1][j - 1]) / (powl(4.0L, (ld)j) - 1.0L);
            grad[q] += (double)R[RICH_LEVELS - 1][RICH_LEVELS - 1];
        }
    }
    free(dcopy);
    return na;
}

/* version tag so the Python side can check the build matches */
int or_abi_version(void) { return 4; }

/* grid length by the points-per-e-fold rule, clamped: N = clamp(ceil(k ln(fmax/fmin)), lo, hi) */
int or_grid_npts(int64_t n, const double *fmin, const double *fmax, double per_efold,
                 int lo, int hi, int32_t *npts)
{
    /* N = ceil(per_efold ln(fmax / fmin)), clamped to [lo, hi]: the definition,
     * in long double */
    for (int64_t e = 0; e < n; e++) {
        ld x = ceill((ld)per_efold * logl((ld)fmax[e] / (ld)fmin[e]));
        if (!(x == x) || x < lo) x = lo;
        if (x > hi) x = hi;
        npts[e] = (int32_t)x;
    }
    return 0;
}
