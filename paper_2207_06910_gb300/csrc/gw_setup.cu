// gw_setup.cu -- per-event kernels around the point loop:
//   catalog preparation (Sec. 2.1, Eq. 2.2, f_ISCO of the Sec. 2.2 footnote),
//   per-event waveform / geometry constants, work-item scan, reduction of the
//   per-item partial sums into SNR / Fisher / VJP outputs, and the batched
//   Cholesky inversion with conditioning check (Sec. 4.1).
#include <cfloat>
#include <cmath>

#include "gw_kernels.cuh"

namespace gw {

// ------------------------------------------------------------------------
// catalog preparation: one thread per event
constexpr double SIX_SQRT6 = 0x1.d64d51e0db1c6p+3;   // 6^(3/2), correctly rounded

__global__ void k_prepare(int64_t n, const double *m1, const double *m2, const double *chi1,
                          const double *chi2, const double *lam1, const double *lam2,
                          const double *dL_Mpc, const uint8_t *zflag, const double *tcoal,
                          const double *fmin, const int32_t *npts_given, int32_t npts_fixed,
                          double per_efold, int32_t lo, int32_t hi, double *Mc, double *eta,
                          double *dL_Gpc, double *chi1o, double *chi2o, double *LamT,
                          double *dLamT, double *tc_s, double *fmax_o, int32_t *npts)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double a = m1[e], b = m2[e], ca = chi1[e], cb = chi2[e];
    double la = lam1 ? lam1[e] : 0.0, lb = lam2 ? lam2[e] : 0.0;
    if (b > a) {   // m1 >= m2, spins and deformabilities follow their body
        double t = a; a = b; b = t;
        t = ca; ca = cb; cb = t;
        t = la; la = lb; lb = t;
    }
    double z = zflag[e] ? H0_KMS_MPC * dL_Mpc[e] / C_KMS : 0.0;
    a *= 1.0 + z;
    b *= 1.0 + z;
    double M = a + b;
    double et = a * b / (M * M);
    double d = (a - b) / M;   // = sqrt(1 - 4 eta) for m1 >= m2, without the cancellation
    double sL = la + lb, dLam = la - lb;
    double lt = 8.0 / 13.0 * ((1.0 + 7.0 * et - 31.0 * et * et) * sL
                              + d * (1.0 + 9.0 * et - 11.0 * et * et) * dLam);
    double dlt = 0.5 * (d * (1.0 - 13272.0 / 1319.0 * et + 8944.0 / 1319.0 * et * et) * sL
                        + (1.0 - 15910.0 / 1319.0 * et + 32850.0 / 1319.0 * et * et
                           + 3380.0 / 1319.0 * et * et * et) * dLam);
    Mc[e] = M * exp(0.6 * log(et));      // eta^(3/5): a few ulp, a fraction of pow's work
    eta[e] = et;
    dL_Gpc[e] = dL_Mpc[e] * 1.0e-3;
    chi1o[e] = ca;
    chi2o[e] = cb;
    LamT[e] = lt;
    dLamT[e] = dlt;
    tc_s[e] = tcoal[e] * T_SIDEREAL;
    double fi = 1.0 / (SIX_SQRT6 * PI * M * T_SUN);   // 1 / (6^(3/2) pi M)
    fmax_o[e] = fi;
    int32_t np;
    if (npts_given) {
        np = npts_given[e];
    } else if (npts_fixed > 0) {
        np = npts_fixed;
    } else {
        double x = ceil(per_efold * log(fi / fmin[e]));
        if (!(x >= (double)lo)) x = lo;   // also catches NaN
        if (x > hi) x = hi;
        np = (int32_t)x;
    }
    npts[e] = np;
}

cudaError_t launch_prepare(int64_t n, const double *m1, const double *m2, const double *chi1,
                           const double *chi2, const double *lam1, const double *lam2,
                           const double *dL_Mpc, const uint8_t *zflag, const double *tcoal,
                           const double *fmin, const int32_t *npts_given, int32_t npts_fixed,
                           double per_efold, int32_t lo, int32_t hi, double *Mc, double *eta,
                           double *dL_Gpc, double *chi1o, double *chi2o, double *LamT,
                           double *dLamT, double *tc_s, double *fmax, int32_t *npts,
                           cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int bs = 256;
    int64_t nb = (n + bs - 1) / bs;
    k_prepare<<<(unsigned)nb, bs, 0, s>>>(n, m1, m2, chi1, chi2, lam1, lam2, dL_Mpc, zflag,
                                          tcoal, fmin, npts_given, npts_fixed, per_efold, lo, hi,
                                          Mc, eta, dL_Gpc, chi1o, chi2o, LamT, dLamT, tc_s, fmax,
                                          npts);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// per-event constants.  TaylorF2 phase and tau* are written in the basis
//   B11 = (v^-5, v^-3, v^-2, v^-1, 1, v, v^2, v^5, v^7, ln v, v ln v)
// at fixed f, so that every parameter derivative is one dot product with the
// point's basis values.  At fixed f:  Mc d/dMc = (1/3) v d/dv  and
// d/deta|Mc = d/deta|v - (1/(5 eta)) v d/dv  (v = (pi M f)^(1/3), M = Mc eta^-3/5).
// constants of the event set-up, as doubles (ln 6, ln 4, pi^(-2/3), sqrt(5/24))
constexpr double LN6 = 0x1.cab0bfa2a2002p+0;
constexpr double LN4 = 0x1.62e42fefa39efp+0;
constexpr double PI_M23 = 0x1.dd61fae9d2f10p-2;
constexpr double SQRT_5_24 = 0x1.d363d1848dcbfp-2;

// (hi, lo) FP32 pair of a double, hi = x rounded to FP32 (nearest, ties to
// even) and lo = x - hi rounded to FP32.  The rounding of hi is done on the bit
// pattern with integer operations, so only the exact difference and the
// conversion of lo use the FP64 pipe (this kernel's bound) instead of three
// conversions and a difference.  Values below FP32's normal range go to lo.
__device__ __forceinline__ float2 split_f32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    // keep 24 significant bits: drop the low 29 of the 52-bit mantissa
    const unsigned long long r = (b + 0x0fffffffull + ((b >> 29) & 1ull)) & ~0x1fffffffull;
    const unsigned ex = (unsigned)(r >> 52) & 0x7ffu;
    if (ex < 1023u - 126u || ex > 1023u + 127u) return make_float2(0.0f, (float)x);
    const unsigned fb = ((unsigned)(r >> 32) & 0x80000000u) | ((ex - 896u) << 23) |
                        ((unsigned)(r >> 29) & 0x7fffffu);
    return make_float2(__uint_as_float(fb), (float)(x - __longlong_as_double((long long)r)));
}

constexpr int SETUP_BS = 128;   // threads per block: two warps per 32 events

__global__ void __launch_bounds__(SETUP_BS)
k_event_setup(DevCat cat, DevNet net, int np, double *evc, double *sitec, float *sitec_f,
              float2 *evc_f, int32_t *status, int64_t *counts, int chunk)
{
    // two warps per 32 events (the set-up is a long chain of dependent FP64
    // operations: twice the warps hide twice the latency): the even warp of a
    // pair writes the status, the scalars and the phase coefficients, the odd
    // one tau* and the per-site constants; each warp follows one path
    const int part = (threadIdx.x >> 5) & 1;
    const int64_t e = ((int64_t)blockIdx.x * (SETUP_BS / 64) + (threadIdx.x >> 6)) * 32 +
                      (threadIdx.x & 31);
    if (e >= cat.n) return;
    const int64_t r = cat.sel ? cat.sel[e] : e;     // catalog row of the call's event e
    const double Mc = cat.Mc[r], eta = cat.eta[r], dL = cat.dL[r];
    const double th = cat.theta[r], ph = cat.phi[r], io = cat.iota[r], ps = cat.psi[r];
    const double tc = cat.tc[r];
    const double c1 = cat.chi1 ? cat.chi1[r] : 0.0, c2 = cat.chi2 ? cat.chi2[r] : 0.0;
    const double LT = cat.LamT ? cat.LamT[r] : 0.0, dLT = cat.dLamT ? cat.dLamT[r] : 0.0;
    const int pset = cat.pset ? (int)cat.pset[r] : 0;
    const double fmin = cat.fmin[r], fmx = cat.fmax[r];
    const int N = cat.npts[r];
    // duty factor: interferometer entries in use for this event's arm mask
    const uint32_t am = cat.arm_mask ? cat.arm_mask[r] : 0xffffffffu;
    uint32_t ifo_on = 0;
    for (int q = 0; q < net.n_ifo; q++) {
        const uint32_t need = net.ifo_need[q], excl = net.ifo_excl[q];
        if ((am & need) == need && !(excl && (am & excl) == excl)) ifo_on |= 1u << q;
    }
    int st = 0;
    if (!(Mc > 0.0) || !(eta > 0.0) || !(eta <= 0.25) || !(dL > 0.0)) st |= 16;
    if (pset < 0 || pset > 2 || ((np == 9) != (pset == 0))) st |= 16;
    if (!isfinite(th) || !isfinite(ph) || !isfinite(io) || !isfinite(ps) || !isfinite(tc) ||
        !isfinite(c1) || !isfinite(c2) || !isfinite(LT) || !isfinite(dLT) ||
        !isfinite(cat.Phic[r]))
        st |= 16;
    if (!(fmin > 0.0) || !(fmx > fmin) || !isfinite(fmx) || N < 2) st |= 8;
    if (part == 0) {
        status[e] = st;
        // no work items when no interferometer is in use (zero SNR and Fisher)
        counts[e] = (st || !ifo_on) ? 0 : (int64_t)((N + chunk - 1) / chunk);
    }
    if (st) return;

    double *E = evc + e * (int64_t)EVC;
    float2 *Ef = evc_f ? evc_f + e * (int64_t)EVC : nullptr;
    const double Mcs = Mc * T_SUN;
    // (x^y as exp(y ln x): a few ulp, at a fraction of pow's FP64 work)
    const double leta = log(eta);
    const double Ms = Mcs * exp(-0.6 * leta);
    const double pi2 = PI * PI;
    const double ie = 1.0 / eta;
    // reciprocals once (the FP64 divide is a multi-instruction sequence)
    const double i3Mc = 1.0 / (3.0 * Mc), i5eta = 0.2 * ie;
    if (part == 0) {
        const double pim = PI * Ms;
        const double lnr = log(fmx / fmin) / (double)(N - 1);
        const double em = expm1(lnr);                 // r - 1, r = f_(k+1) / f_k
        const double emn = em / (1.0 + em);           // 1 - 1/r
        E[EV_MC] = Mc;
        E[EV_ETA] = eta;
        E[EV_DL] = dL;
        E[EV_NPTS] = (double)N;
        E[EV_LNR] = lnr;
        E[EV_WC0] = 0.5 * em;
        E[EV_WCM] = 0.5 * em + 0.5 * emn;            // sinh(ln r) = (r - 1/r) / 2
        E[EV_WCN] = 0.5 * emn;
        E[EV_LNF0] = log(fmin);
        E[EV_LNPIM] = log(pim);
        E[EV_INV_PIM] = 1.0 / pim;
        E[EV_PIM] = pim;
        const double rhog = exp(GROUP * lnr / 3.0);
        E[EV_RHOG] = rhog;
        E[EV_RHOIG] = 1.0 / rhog;
        E[EV_LNRHOG] = GROUP * lnr / 3.0;
        E[EV_A0] = SQRT_5_24 * PI_M23 * exp(5.0 / 6.0 * log(Mcs)) / (dL * GPC_S);
        E[EV_RAG] = exp(-7.0 / 6.0 * GROUP * lnr);
        for (int g = 0; g < 2; g++) {        // the same over 4 and over 16 points
            const double L = (g == 0 ? 4.0 : 16.0) * lnr;
            const double rg = exp(L / 3.0);
            E[EV_ADV + 4 * g] = rg;
            E[EV_ADV + 4 * g + 1] = 1.0 / rg;
            E[EV_ADV + 4 * g + 2] = L / 3.0;
            E[EV_ADV + 4 * g + 3] = exp(-7.0 / 6.0 * L);
        }
        double si, ci, s2p, c2p;
        sincos(io, &si, &ci);
        sincos(2.0 * ps, &s2p, &c2p);
        E[EV_CP] = 0.5 * (1.0 + ci * ci);
        E[EV_CX] = ci;
        E[EV_DCP] = -ci * si;
        E[EV_DCX] = -si;
        E[EV_C2PSI] = c2p;
        E[EV_S2PSI] = s2p;
        E[EV_AMC] = 5.0 / (6.0 * Mc);
        E[EV_INVDL] = 1.0 / dL;
        E[EV_IFOON] = (double)ifo_on;
        E[EV_ARMON] = (double)am;
        E[EV_PHI0] = -cat.Phic[r] - 0.25 * PI;

        // ---- TaylorF2 3.5PN phase coefficients (restricted PN)
        const double d = sqrt(fmax(0.0, 1.0 - 4.0 * eta));
        const double X1 = 0.5 * (1.0 + d), X2 = 0.5 * (1.0 - d);
        const double b1 = 113.0 / 12.0 * X1 * X1 + 25.0 * eta / 4.0;
        const double b2 = 113.0 / 12.0 * X2 * X2 + 25.0 * eta / 4.0;
        const double beta = b1 * c1 + b2 * c2;
        const double sigma = 79.0 / 8.0 * eta * c1 * c2;
        const double dbeta = 113.0 / 6.0 * (X2 * c2 - X1 * c1) / d + 25.0 / 4.0 * (c1 + c2);
        const double dsigma = 79.0 / 8.0 * c1 * c2;
        const double ln6h = 1.0 + 1.5 * LN6;                      // 1 - 3 ln v_lso
        const double L6 = -6848.0 / 21.0;
        const double p2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
        const double p3 = -16.0 * PI + 4.0 * beta;
        const double p4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta
                          - 10.0 * sigma;
        const double p5a = PI * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
        const double p5c = p5a * ln6h;
        const double p6c = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2
                           - 6848.0 / 21.0 * EULER_GAMMA
                           + (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) * eta
                           + 76055.0 / 1728.0 * eta * eta - 127825.0 / 1296.0 * eta * eta * eta;
        const double p6 = p6c + L6 * LN4;
        const double p7 = PI * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta
                                - 74045.0 / 756.0 * eta * eta);
        const double t10 = -39.0 / 2.0 * LT;
        const double t12 = -3115.0 / 64.0 * LT + 6595.0 / 364.0 * d * dLT;
        const double dp4 = 27145.0 / 504.0 + 2.0 * 3085.0 / 72.0 * eta - 10.0 * dsigma;
        const double dp5a = -65.0 * PI / 9.0;
        const double dp6 = -15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2
                           + 2.0 * 76055.0 / 1728.0 * eta - 3.0 * 127825.0 / 1296.0 * eta * eta;
        const double dp7 = PI * (378515.0 / 1512.0 - 2.0 * 74045.0 / 756.0 * eta);
        const double dt12 = 6595.0 / 364.0 * (-2.0 / d) * dLT;
        const double pre = 3.0 / 128.0 * ie;
        // v dPsi/dv
        const double V[11] = {-5.0, -3.0 * p2, -2.0 * p3, -p4, 3.0 * p5a, p6 + L6, 2.0 * p7,
                              5.0 * t10, 7.0 * t12, 0.0, L6};
        // dPsi/deta at fixed v (before the prefactor)
        const double De[11] = {-ie, 55.0 / 9.0 - p2 * ie, 4.0 * dbeta - p3 * ie, dp4 - p4 * ie,
                               dp5a * ln6h - p5c * ie, dp6 - p6 * ie, dp7 - p7 * ie, -t10 * ie,
                               dt12 - t12 * ie, 3.0 * (dp5a - p5a * ie), -L6 * ie};
        // Psi itself (strain output): v^-5 (1, p2 v^2, p3 v^3, p4 v^4) + p5a (1 - 3 ln v_lso
        // + 3 ln v) + (p6 + L6 ln v) v + p7 v^2 + tidal v^5, v^7, all times 3/(128 eta)
        const double Ps[11] = {1.0, p2, p3, p4, p5c, p6, p7, t10, t12, 3.0 * p5a, L6};
        for (int k = 0; k < 11; k++) {
            E[EV_PSI + k] = pre * Ps[k];
            E[EV_PM + k] = pre * V[k] * i3Mc;
            E[EV_PE + k] = pre * (De[k] - V[k] * i5eta);
        }
        double q9[4] = {0, 0, 0, 0}, q10[4] = {0, 0, 0, 0};
        if (pset == 1) {
            q9[0] = 4.0 * b1;
            q9[1] = -10.0 * 79.0 / 8.0 * eta * c2;
            q10[0] = 4.0 * b2;
            q10[1] = -10.0 * 79.0 / 8.0 * eta * c1;
        } else if (pset == 2) {
            q9[2] = -39.0 / 2.0;
            q9[3] = -3115.0 / 64.0;
            q10[3] = 6595.0 / 364.0 * d;
        }
        for (int k = 0; k < 4; k++) {
            E[EV_P9 + k] = pre * q9[k];
            E[EV_P10 + k] = pre * q10[k];
        }
        // double-float (hi, lo) copy of the constants the mixed point loop reads
        // (slots EV_WC0 .. EV_INVDL and the polynomial coefficients EV_PM ..)
        if (Ef) {
            for (int q = EV_WC0; q < EV_T0; q++) {
                if (q > EV_INVDL && q < EV_PM) continue;
                Ef[q] = split_f32(E[q]);
            }
            for (int q = EV_ADV; q < EVC; q++) Ef[q] = split_f32(E[q]);
        }
    } else {
        // ---- tau*(f), 3.5PN (Buonanno et al. 2009 Eq. 3.8b), basis B8 times v^-3
        const double Kt = 5.0 * Ms / (256.0 * eta);
        const double t2 = 743.0 / 252.0 + 11.0 / 3.0 * eta;
        const double t3 = -32.0 / 5.0 * PI;
        const double t4 = 3058673.0 / 508032.0 + 5429.0 / 504.0 * eta + 617.0 / 72.0 * eta * eta;
        const double t5 = (-7729.0 / 252.0 + 13.0 / 3.0 * eta) * PI;
        const double t6 = -10052469856691.0 / 23471078400.0 + 128.0 / 3.0 * pi2
                          + 6848.0 / 105.0 * EULER_GAMMA
                          + (3147553127.0 / 3048192.0 - 451.0 / 12.0 * pi2) * eta
                          - 15211.0 / 1728.0 * eta * eta + 25565.0 / 1296.0 * eta * eta * eta
                          + 3424.0 / 105.0 * (2.0 * LN4);
        const double t6L = 6848.0 / 105.0;
        const double t7 = (-15419335.0 / 127008.0 - 75703.0 / 756.0 * eta
                           + 14809.0 / 378.0 * eta * eta) * PI;
        const double dt4 = 5429.0 / 504.0 + 2.0 * 617.0 / 72.0 * eta;
        const double dt5 = 13.0 / 3.0 * PI;
        const double dt6 = 3147553127.0 / 3048192.0 - 451.0 / 12.0 * pi2
                           - 2.0 * 15211.0 / 1728.0 * eta + 3.0 * 25565.0 / 1296.0 * eta * eta;
        const double dt7 = PI * (-75703.0 / 756.0 + 2.0 * 14809.0 / 378.0 * eta);
        const double T0[8] = {1.0, t2, t3, t4, t5, t6, t7, t6L};
        const double Tv[8] = {-5.0, -3.0 * t2, -2.0 * t3, -t4, 0.0, t6 + t6L, 2.0 * t7, t6L};
        const double Te[8] = {-ie, 11.0 / 3.0 - t2 * ie, -t3 * ie, dt4 - t4 * ie, dt5 - t5 * ie,
                              dt6 - t6 * ie, dt7 - t7 * ie, -t6L * ie};
        for (int k = 0; k < 8; k++) {
            E[EV_T0 + k] = Kt * T0[k];
            E[EV_TM + k] = Kt * Tv[k] * i3Mc;
            E[EV_TE + k] = Kt * (Te[k] - Tv[k] * i5eta);
        }

        if (Ef)
            for (int q = EV_T0; q < EV_COEF_END; q++) Ef[q] = split_f32(E[q]);

        // ---- per-site JKS coefficients (pattern functions as functions of the
        // hour-angle-like x = phi - lon - g) and Doppler factors.
        double sth, cth;
        sincos(th, &sth, &cth);
        const double sd = cth, cd = sth;                  // delta = pi/2 - theta
        const double s2d = 2.0 * sth * cth, c2d = sth * sth - cth * cth;
        for (int s = 0; s < net.n_site; s++) {
            double *S = sitec + (e * net.n_site + s) * (int64_t)SC_N;
            const double sl = net.site_slat[s], cl = net.site_clat[s];
            const double c2l = 1.0 - 2.0 * sl * sl, s2l = 2.0 * sl * cl;
            double x0 = ph - net.site_lon[s] - OMEGA_E * tc;
            // x0 - 2 pi round(x0 / 2 pi): the FMA forms n 2 pi exactly and the
            // difference (at most ~pi in magnitude) is representable, so this is
            // exactly remainder(x0, 2 pi) up to the choice at +-pi
            x0 = fma(-rint(x0 * (1.0 / TWO_PI)), TWO_PI, x0);
            S[SC_X0] = x0;
            S[SC_A1] = (3.0 - c2l) * (3.0 - c2d) / 16.0;
            S[SC_A2] = s2l * s2d / 4.0;
            S[SC_A3] = 0.75 * cl * cl * cd * cd;
            S[SC_A4] = -sl * (3.0 - c2d) / 4.0;
            S[SC_A5] = -cl * s2d / 2.0;
            S[SC_B1] = sl * sd;
            S[SC_B2] = cl * cd;
            S[SC_B3] = (3.0 - c2l) * sd / 4.0;
            S[SC_B4] = s2l * cd / 2.0;
            // d/dtheta = -d/ddelta
            S[SC_A1T] = -(3.0 - c2l) * s2d / 8.0;
            S[SC_A2T] = -s2l * c2d / 2.0;
            S[SC_A3T] = 0.75 * cl * cl * s2d;
            S[SC_A4T] = sl * s2d / 2.0;
            S[SC_A5T] = cl * c2d;
            S[SC_B1T] = -sl * cd;
            S[SC_B2T] = cl * sd;
            S[SC_B3T] = -(3.0 - c2l) * cd / 4.0;
            S[SC_B4T] = s2l * sd / 2.0;
            S[SC_D1] = R_EARTH_S * cl * sth;
            S[SC_D2] = R_EARTH_S * sl * cth;
            S[SC_D1T] = R_EARTH_S * cl * cth;
            S[SC_D2T] = -R_EARTH_S * sl * sth;
            // the (at most two) interferometer entries of this site in use: the
            // point kernels run a fixed number of slots per site, whatever the mask
            int slot[2] = {-1, -1}, nsl = 0;
            for (int q = net.site_ifo0[s]; q < net.site_ifo1[s] && nsl < 2; q++)
                if ((ifo_on >> q) & 1u) slot[nsl++] = q;
            S[SC_SLOT0] = (double)slot[0];
            S[SC_SLOT1] = (double)slot[1];
            S[SC_X0LO] = 0.0;
            if (sitec_f) {
                float *Sf = sitec_f + (e * net.n_site + s) * (int64_t)SC_N;
                // (float)S[q]: hi, or lo where the value is below FP32's normal range
                for (int q = 0; q < SC_N; q++) {
                    const float2 v = split_f32(S[q]);
                    Sf[q] = v.x != 0.0f ? v.x : v.y;
                }
                const float2 xs = split_f32(x0);
                Sf[SC_X0] = xs.x != 0.0f ? xs.x : xs.y;
                Sf[SC_X0LO] = xs.x != 0.0f ? xs.y : 0.0f;
            }
        }
    }
}

cudaError_t launch_event_setup(const DevCat &cat, const DevNet &net, int np, double *evc,
                               double *sitec, float *sitec_f, float2 *evc_f, int32_t *status,
                               int64_t *counts, cudaStream_t s, int chunk)
{
    if (cat.n <= 0) return cudaSuccess;
    const int64_t per_block = SETUP_BS / 2;       // events per block
    const int64_t nb = (cat.n + per_block - 1) / per_block;
    k_event_setup<<<(unsigned)nb, SETUP_BS, 0, s>>>(cat, net, np, evc, sitec, sitec_f, evc_f,
                                                   status, counts, chunk);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// exclusive scan (int64), three passes: block sums, scan of block sums in one
// block, then per-block offsets.  SCAN_BS elements per block.
constexpr int SCAN_BS = 1024;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ int64_t block_excl_scan(int64_t v, int64_t &excl)
{
    __shared__ int64_t wsum[SCAN_BS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t x = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        x = warp_incl_scan(x);
        if (lane < (int)(blockDim.x >> 5)) wsum[lane] = x;
    }
    __syncthreads();
    int64_t base = (w > 0) ? wsum[w - 1] : 0;
    excl = base + inc - v;
    int64_t total = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return total;
}

__global__ void k_scan_blocks(const int64_t *counts, int64_t n, int64_t *off, int64_t *bsum)
{
    int64_t i = blockIdx.x * (int64_t)SCAN_BS + threadIdx.x;
    int64_t v = (i < n) ? counts[i] : 0;
    int64_t ex;
    int64_t tot = block_excl_scan(v, ex);
    if (i < n) off[i] = ex;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t *bsum, int64_t nb, int64_t *off_total)
{
    // single block; loops over chunks of SCAN_BS block sums
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_BS) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = (i < nb) ? bsum[i] : 0;
        int64_t ex;
        int64_t tot = block_excl_scan(v, ex);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *off_total = carry;
}

__global__ void k_scan_add(int64_t *off, int64_t n, const int64_t *bsum)
{
    int64_t i = blockIdx.x * (int64_t)SCAN_BS + threadIdx.x;
    if (i < n) off[i] += bsum[blockIdx.x];
}

size_t scan_tmp_size(int64_t n) { return (size_t)((n + SCAN_BS - 1) / SCAN_BS + 1); }

cudaError_t launch_scan(const int64_t *counts, int64_t n, int64_t *off, int64_t *tmp,
                        cudaStream_t s)
{
    int64_t nb = (n + SCAN_BS - 1) / SCAN_BS;
    if (nb < 1) nb = 1;
    k_scan_blocks<<<(unsigned)nb, SCAN_BS, 0, s>>>(counts, n, off, tmp);
    k_scan_sums<<<1, SCAN_BS, 0, s>>>(tmp, nb, off + n);
    k_scan_add<<<(unsigned)nb, SCAN_BS, 0, s>>>(off, n, tmp);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// reduction of item partials: one block per tile of FIN_EV consecutive events.
// Their items are consecutive rows of `partial`, so the block reads one
// contiguous span (accumulator fastest) and sums each event's items in item
// order (deterministic) into shared memory; every output row is then written
// as one coalesced run of FIN_EV events (the outputs are event-minor).
constexpr int FIN_EV = 32;
constexpr int FIN_BS = 256;

__global__ void __launch_bounds__(FIN_BS) k_finish(int mode, int np, int n_det, int64_t n,
                                                   int nacc, int64_t cap,
                                                   const int64_t *item_off,
                                                   const double *partial, int32_t *status,
                                                   double *snr, double *snr_det, double *fisher,
                                                   const double *grad_snr, double *grad_params,
                                                   double *xsums)
{
    extern __shared__ double fin_s[];     // [nacc][FIN_EV + 1]
    constexpr int LD = FIN_EV + 1;
    const int64_t e0 = blockIdx.x * (int64_t)FIN_EV;
    const int ne = (int)(n - e0 < FIN_EV ? n - e0 : FIN_EV);
    for (int q = threadIdx.x; q < ne * nacc; q += FIN_BS) {
        const int le = q / nacc, a = q - le * nacc;
        const int64_t i0 = item_off[e0 + le], i1 = item_off[e0 + le + 1];
        double s = 0.0;
        if (i1 <= cap)                    // items beyond the workspace capacity: none
            for (int64_t it = i0; it < i1; it++) s += partial[it * nacc + a];
        fin_s[a * LD + le] = s;
    }
    __syncthreads();
    const int npair = np * (np + 1) / 2;
    for (int q = threadIdx.x; q < nacc * FIN_EV; q += FIN_BS) {
        const int a = q / FIN_EV, le = q - a * FIN_EV;
        if (le >= ne) continue;
        const int64_t e = e0 + le;
        const bool over = item_off[e + 1] > cap;
        if (over && a == 0) status[e] |= 64;
        const bool bad = over || (status[e] & ~64) != 0;
        const double s = fin_s[a * LD + le];
        if (mode == MODE_FISHER) {
            if (a == 0) {
                if (snr) snr[e] = bad ? NAN : sqrt(s);
            } else if (a <= npair) {
                fisher[(int64_t)(a - 1) * n + e] = bad ? NAN : s;
            } else if (xsums) {
                xsums[(int64_t)(a - 1 - npair) * n + e] = bad ? NAN : s;
            }
        } else if (mode == MODE_SNR) {
            if (a == 0) snr[e] = bad ? NAN : sqrt(s);
            else if (snr_det) snr_det[(int64_t)(a - 1) * n + e] = bad ? NAN : sqrt(s);
        } else if (mode == MODE_SNRGRAD) {
            if (a > 0) {
                const double s0 = fin_s[le];
                // d SNR / d theta = sum W Re(Q* g) / SNR (zero when no arm is on)
                const double g = s0 > 0.0 ? grad_snr[e] * s / sqrt(s0) : 0.0;
                if (a <= np) grad_params[(int64_t)(a - 1) * n + e] = bad ? NAN : g;
                // detector orientations: the event's term of the sum over events
                // (flagged events left out of the sum)
                else if (xsums) xsums[(int64_t)(a - 1 - np) * n + e] = bad ? 0.0 : g;
            }
        }
    }
}

// Log table of a tabulated noise curve (Sec. 3.1, the psd_path / is_ASD
// options): segment j holds ln f_j, ln S_j (S = scale x table value, the value
// squared for an amplitude spectral density), the slope of ln S over ln f to
// the next node, and ln f_j+1; the mixed path's copy holds ln f and
// ln S - ln(reference scale) as double-float pairs.  One block per table: if
// any entry breaks the table's rules (f > 0 strictly increasing, values > 0,
// all finite), every segment's ln S is NaN, so every noise weight is NaN.
__global__ void __launch_bounds__(256) k_psd_table(const double *f, const double *S, int64_t nseg,
                                                   int is_asd, double ln_scale, double ln_ref,
                                                   PsdSeg *seg, float4 *segf)
{
    int ok = 1;
    for (int64_t j = threadIdx.x; j < nseg; j += blockDim.x) {
        const double f0 = f[j], f1 = f[j + 1], s0 = S[j], s1 = S[j + 1];
        ok &= f0 > 0.0 && f1 > f0 && isfinite(f1) && s0 > 0.0 && s1 > 0.0 && isfinite(s0) &&
              isfinite(s1);
    }
    ok = __syncthreads_and(ok);
    const double pw = is_asd ? 2.0 : 1.0;
    for (int64_t j = threadIdx.x; j < nseg; j += blockDim.x) {
        const double lf0 = log(f[j]), lf1 = log(f[j + 1]);
        double ls0 = fma(pw, log(S[j]), ln_scale);
        const double ls1 = fma(pw, log(S[j + 1]), ln_scale);
        double slope = (ls1 - ls0) / (lf1 - lf0);
        if (!ok) ls0 = slope = NAN;
        seg[j] = PsdSeg{lf0, ls0, slope, lf1};
        if (segf) {
            const double rel = ls0 - ln_ref;
            const float a = (float)lf0, b = (float)rel, c = (float)lf1;
            segf[2 * j] = make_float4(a, (float)(lf0 - (double)a), b, (float)(rel - (double)b));
            segf[2 * j + 1] = make_float4((float)slope, c, (float)(lf1 - (double)c), 0.0f);
        }
    }
}

cudaError_t launch_psd_table(const double *f, const double *S, int64_t nseg, int is_asd,
                             double ln_scale, double ln_ref, PsdSeg *seg, float4 *segf,
                             cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    k_psd_table<<<1, 256, 0, s>>>(f, S, nseg, is_asd, ln_scale, ln_ref, seg, segf);
    return cudaGetLastError();
}

// detection gate (snr_th): flags, then order-preserving compaction after an
// exclusive scan of the flags
__global__ void k_flag_gt(const double *snr, int64_t n, double th, int64_t *flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = snr[i] > th ? 1 : 0;
}

__global__ void k_compact(const double *snr, int64_t n, double th, const int64_t *off,
                          int64_t *sel)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && snr[i] > th) sel[off[i]] = i;
}

cudaError_t launch_select(const double *snr, int64_t n, double th, int64_t *flag, int64_t *off,
                          int64_t *scan_tmp, int64_t *sel, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int bs = 256;
    const unsigned nb = (unsigned)((n + bs - 1) / bs);
    k_flag_gt<<<nb, bs, 0, s>>>(snr, n, th, flag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_scan(flag, n, off, scan_tmp, s)) != cudaSuccess) return e;
    k_compact<<<nb, bs, 0, s>>>(snr, n, th, off, sel);
    return cudaGetLastError();
}

// sum over events of each row of x [rows][n], fixed order
__global__ void k_sum_events(const double *x, int64_t n, double *out)
{
    __shared__ double sh[256];
    const int r = blockIdx.x;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += x[(int64_t)r * n + e];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r] = sh[0];
}

cudaError_t launch_sum_events(const double *x, int64_t n, int rows, double *out, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_sum_events<<<rows, 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

// logdet mode: total over all items of each detector accumulator, fixed order
__global__ void k_finish_total(int64_t cap, const int64_t *total, int nacc, const double *partial,
                               uint32_t det_mask, double *out)
{
    __shared__ double sh[256];
    const int64_t n_items = *total < cap ? *total : cap;
    int a = blockIdx.x;
    double s = 0.0;
    for (int64_t it = threadIdx.x; it < n_items; it += blockDim.x) s += partial[it * nacc + a];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[a] = (det_mask >> a) & 1u ? sh[0] : NAN;   // NaN: not requested
}

// SNR vector-Jacobian product after a Fisher pass, one thread per event.
//  FP64 path: d SNR/d theta_i = -dL Gamma_{i,dL} / SNR, because d h/d dL = -h/dL
//             makes Re(h^* d_i h) = -dL Re(d_dL h^* d_i h) (Sec. 3.2 definitions).
//  mixed path: phase-free sums (the phase part of Re(h^* d_i h) is zero):
//             Mc: 5/(6 Mc) SNR^2 + X1, eta: X2, dL: -SNR^2/dL, theta: X3, phi: X0,
//             iota: X4, psi: X5, tc: -Omega_E X0, Phic and slots 9, 10: 0.
__global__ void k_snr_grad(int64_t n, int np, int mixed, int rot, const double *F,
                           const double *snr, const double *X, const double *evc,
                           const int32_t *status, const double *grad_snr, double *grad)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const bool bad = status[e] != 0;
    const double s = snr[e], up = grad_snr[e];
    const double d = evc[e * (int64_t)EVC + EV_DL], Mc = evc[e * (int64_t)EVC + EV_MC];
    for (int i = 0; i < np; i++) {
        double g;
        if (!(s > 0.0)) {
            g = 0.0;   // no arm on (duty factor): the SNR is identically zero
        } else if (!mixed) {
            const int lo = i < 2 ? i : 2, hi = i < 2 ? 2 : i;
            const int k = lo * np - lo * (lo - 1) / 2 + (hi - lo);
            g = -d * F[(int64_t)k * n + e] / s;
        } else {
            const double s2 = s * s;
            switch (i) {
            case 0: g = (5.0 / (6.0 * Mc) * s2 + X[1 * n + e]) / s; break;
            case 1: g = X[2 * n + e] / s; break;
            case 2: g = -s2 / (d * s); break;
            case 3: g = X[3 * n + e] / s; break;
            case 4: g = X[0 * n + e] / s; break;
            case 5: g = X[4 * n + e] / s; break;
            case 6: g = X[5 * n + e] / s; break;
            case 7: g = rot ? -OMEGA_E * X[0 * n + e] / s : 0.0; break;   // tc moves x only with rotation
            default: g = 0.0;
            }
        }
        grad[(int64_t)i * n + e] = bad ? NAN : up * g;
    }
}

cudaError_t launch_snr_grad_from_fisher(int64_t n, int np, bool mixed, int rot,
                                        const double *fisher, const double *snr,
                                        const double *xsums, const double *evc,
                                        const int32_t *status, const double *grad_snr,
                                        double *grad_params, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int bs = 256;
    k_snr_grad<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(n, np, mixed ? 1 : 0, rot, fisher, snr,
                                                            xsums, evc, status, grad_snr,
                                                            grad_params);
    return cudaGetLastError();
}

cudaError_t launch_finish(int mode, int np, int n_det, const PointArgs &a, const int32_t *status,
                          double *snr, double *snr_det, double *fisher, const double *grad_snr,
                          double *grad_params, double *grad_gamma, double *xsums, cudaStream_t s)
{
    if (mode == MODE_LOGDET) {
        k_finish_total<<<a.nacc, 256, 0, s>>>(a.n_items, a.item_off + a.n_ev, a.nacc, a.partial,
                                              a.det_mask, grad_gamma);
        return cudaGetLastError();
    }
    if (a.n_ev <= 0 || a.nacc <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.nacc * (FIN_EV + 1) * sizeof(double);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    k_finish<<<(unsigned)((a.n_ev + FIN_EV - 1) / FIN_EV), FIN_BS, smem, s>>>(
        mode, np, n_det, a.n_ev, a.nacc, a.n_items, a.item_off, a.partial,
        const_cast<int32_t *>(status), snr, snr_det, fisher, grad_snr, grad_params, xsums);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Batched inversion (Sec. 4.1): normalise by sqrt(diag), Cholesky, triangular
// inverse, C = L^-T L^-1 rescaled; 1-norm condition number of the normalised
// matrix and eps = max |Gamma C - 1|.  One thread per event, FP64.  Everything
// happens in place on one packed lower triangle (H, then L, then M = L^-1,
// then C), so that a thread holds P(P+1)/2 values; the rows of Gamma for eps
// are read again from the input.
template <int NP>
__device__ __forceinline__ constexpr int pkt(int i, int j)   // packed upper (i <= j)
{
    return i * NP - i * (i - 1) / 2 + (j - i);
}

__device__ __forceinline__ constexpr int plt(int i, int j)   // packed lower (j <= i)
{
    return i * (i + 1) / 2 + j;
}

template <int NP>
__global__ void __launch_bounds__(128) k_invert(const double *F, int64_t n, double cond_max,
                                                double *cov, double *cond, double *inv_err,
                                                int32_t *status)
{
    constexpr int NK = NP * (NP + 1) / 2;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double T[NK];           // lower triangle: H, then L, then M = L^-1, then C
    double id[NP], il[NP];
    int st = 0;
    // (the FP64 pipe is this kernel's bound: tests on the bit patterns go to
    // the integer pipe, and one reciprocal square root replaces each
    // square root and divide)
    unsigned nonfin = 0;
#pragma unroll
    for (int i = 0; i < NP; i++)
#pragma unroll
        for (int j = 0; j < NP; j++) {
            if (j < i) continue;
            const double v = F[(int64_t)pkt<NP>(i, j) * n + e];
            nonfin |= ((unsigned)(__double_as_longlong(v) >> 52) & 0x7ffu) == 0x7ffu;
            T[plt(j, i)] = v;
        }
    if (nonfin) st |= 4;
#pragma unroll
    for (int i = 0; i < NP; i++) {
        if (!(T[plt(i, i)] > 0.0)) st |= 1;
        id[i] = rsqrt(T[plt(i, i)]);   // 1 / sqrt(Gamma_ii)
    }
    double kappa = NAN, eps = NAN;
    if (!st) {
        // normalise, and the 1-norm of H (symmetric: column sums from the lower triangle)
        double colh[NP];
#pragma unroll
        for (int j = 0; j < NP; j++) colh[j] = 0.0;
#pragma unroll
        for (int i = 0; i < NP; i++)
#pragma unroll
            for (int j = 0; j < NP; j++) {
                if (j > i) continue;
                T[plt(i, j)] *= id[i] * id[j];
                colh[j] += fabs(T[plt(i, j)]);
                if (i != j) colh[i] += fabs(T[plt(i, j)]);
            }
        double hn1 = 0.0;
#pragma unroll
        for (int j = 0; j < NP; j++) hn1 = fmax(hn1, colh[j]);
        // Cholesky H = L L^T in place (the diagonal of L is kept as 1 / L_jj only)
#pragma unroll
        for (int j = 0; j < NP; j++) {
            double sjj = T[plt(j, j)];
#pragma unroll
            for (int k = 0; k < NP; k++)
                if (k < j) sjj -= T[plt(j, k)] * T[plt(j, k)];
            if (!(sjj > 0.0)) st |= 1;
            il[j] = rsqrt(sjj);
#pragma unroll
            for (int i = 0; i < NP; i++) {
                if (i <= j) continue;
                double t = T[plt(i, j)];
#pragma unroll
                for (int k = 0; k < NP; k++)
                    if (k < j) t -= T[plt(i, k)] * T[plt(j, k)];
                T[plt(i, j)] = t * il[j];
            }
        }
        if (!st) {
            // M = L^-1 in place, column by column from the left: M_ij =
            // -(1/L_ii) sum_{k=j}^{i-1} L_ik M_kj reads L only in columns >= j
            // of rows > i-1, which are still L
#pragma unroll
            for (int j = 0; j < NP; j++) {
                T[plt(j, j)] = il[j];
#pragma unroll
                for (int i = 0; i < NP; i++) {
                    if (i <= j) continue;
                    double t = 0.0;
#pragma unroll
                    for (int k = 0; k < NP; k++)
                        if (k >= j && k < i) t = fma(T[plt(i, k)], T[plt(k, j)], t);
                    T[plt(i, j)] = -t * il[i];
                }
            }
            // Hinv = M^T M in place, row by row from the top: Hinv_ij (j <= i)
            // = sum_{k>=i} M_ki M_kj reads rows >= i of M only, and of row i
            // only M_ii and M_ij, so the diagonal entry is written last.  Its
            // 1-norm, then the rescaled C = D^-1 Hinv D^-1 in place.
            double coli[NP];
#pragma unroll
            for (int j = 0; j < NP; j++) coli[j] = 0.0;
#pragma unroll
            for (int i = 0; i < NP; i++) {
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    if (j >= i) continue;
                    double t = 0.0;
#pragma unroll
                    for (int k = 0; k < NP; k++)
                        if (k >= i) t = fma(T[plt(k, i)], T[plt(k, j)], t);
                    coli[j] += fabs(t);
                    coli[i] += fabs(t);
                    T[plt(i, j)] = t;
                }
                double t = 0.0;
#pragma unroll
                for (int k = 0; k < NP; k++)
                    if (k >= i) t = fma(T[plt(k, i)], T[plt(k, i)], t);
                coli[i] += fabs(t);
                T[plt(i, i)] = t;
            }
            double in1 = 0.0;
#pragma unroll
            for (int j = 0; j < NP; j++) in1 = fmax(in1, coli[j]);
#pragma unroll
            for (int i = 0; i < NP; i++)
#pragma unroll
                for (int j = 0; j < NP; j++)
                    if (j <= i) T[plt(i, j)] *= id[i] * id[j];
            kappa = hn1 * in1;
            if (kappa > 1.0 / DBL_EPSILON) st |= 32;
            if (kappa > cond_max) st |= 2;
            if (inv_err) {
                // eps = max |Gamma C - 1|, Gamma row by row from the input; the
                // maximum of |t| on the bit patterns (ordered as unsigned
                // integers for finite doubles once the sign bit is cleared)
                unsigned long long emax = 0;
#pragma unroll
                for (int i = 0; i < NP; i++) {
                    // (keeps the compiler from loading every row of Gamma at once)
                    asm volatile("" ::: "memory");
                    double g[NP];
#pragma unroll
                    for (int k = 0; k < NP; k++)
                        g[k] = F[(int64_t)pkt<NP>(i < k ? i : k, i < k ? k : i) * n + e];
#pragma unroll
                    for (int j = 0; j < NP; j++) {
                        double t = (i == j) ? -1.0 : 0.0;
#pragma unroll
                        for (int k = 0; k < NP; k++)
                            t = fma(g[k], T[k > j ? plt(k, j) : plt(j, k)], t);
                        const unsigned long long tb =
                            (unsigned long long)__double_as_longlong(t) & 0x7fffffffffffffffull;
                        emax = tb > emax ? tb : emax;
                    }
                }
                eps = __longlong_as_double((long long)emax);
            }
        }
    }
    const bool ok = !(st & (1 | 2 | 4));
#pragma unroll
    for (int i = 0; i < NP; i++)
#pragma unroll
        for (int j = 0; j < NP; j++)
            if (j >= i) cov[(int64_t)pkt<NP>(i, j) * n + e] = ok ? T[plt(j, i)] : NAN;
    if (cond) cond[e] = (st & (1 | 4)) ? NAN : kappa;
    if (inv_err) inv_err[e] = ok ? eps : NAN;
    status[e] = st;
}

cudaError_t launch_invert(const double *fisher, int64_t n, int np, double cond_max, double *cov,
                          double *cond, double *inv_err, int32_t *status, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    // one warp per block: at ~255 registers a thread, eight warps fit an SM
    // either way, and a small call (the events a refinement recomputes)
    // spreads over twice as many SMs as with blocks of two warps
    int bs = 32;
    unsigned nb = (unsigned)((n + bs - 1) / bs);
    if (np == 9)
        k_invert<9><<<nb, bs, 0, s>>>(fisher, n, cond_max, cov, cond, inv_err, status);
    else
        k_invert<11><<<nb, bs, 0, s>>>(fisher, n, cond_max, cov, cond, inv_err, status);
    return cudaGetLastError();
}

}  // namespace gw
