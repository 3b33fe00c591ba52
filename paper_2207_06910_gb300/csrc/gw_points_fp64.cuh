// gw_points_fp64.cuh -- the fused point loop, every operation in FP64.
//
// One group of G lanes (8 by default) per work item (a contiguous run of at most CHUNK_MAX
// grid points of one event); lane l of the group takes points k0 + l,
// k0 + l + G, ...  For each point it
// forms the TaylorF2 phase derivatives, tau*(f) and its derivatives (Sec. 2.2),
// the pattern functions and Doppler phase at the Earth angle of t(f)
// (Sec. 3.1), the tangents g_i = dQ/dtheta_i + i Q dPhi/dtheta_i of every
// (virtual) interferometer and accumulates
//     SNR^2 += W |Q|^2,   Gamma_ij += W Re(g_i^* g_j),   W = 4 w_k / S_n(f_k)
// (Sec. 3.2, Eqs. 3.1-3.3, trapezoid weights w_k on the log grid).  The strain
// phase Phi itself is never formed: with h = Q e^{i Phi} the factor e^{i Phi}
// cancels in |h|^2 and in Re(d_i h^* d_j h), so only its derivatives enter.
// Tangents never leave registers; each group writes one row of partial sums.
#pragma once

#include <cmath>
#include <type_traits>

#include "gw_kernels.cuh"
#include "gw_dfloat.cuh"

namespace gw {

namespace {

// reciprocal: hardware estimate refined by two Newton-Raphson steps
// y <- y (2 - x y) (Newton's method for f(y) = 1/y - x)
__device__ __forceinline__ double rcp64(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    return y;
}

__device__ __forceinline__ double ipow(double x, int p)
{
    double r = 1.0;
    while (p) {
        if (p & 1) r *= x;
        x *= x;
        p >>= 1;
    }
    return r;
}

__device__ __forceinline__ int64_t find_event(const int64_t *off, int64_t n, int64_t it)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int MODE, int NP>
struct NAccOf {
    static constexpr int value = MODE == MODE_FISHER ? 1 + NP * (NP + 1) / 2
                               : MODE == MODE_SNRGRAD ? 1 + NP + MAX_DET
                               : MODE == MODE_SNR ? 1 + MAX_DET
                               : MAX_DET;
};

// per-IFO pattern values at one point
// (T: double on the FP64 pipe, dfl in double-float on the FP32 pipe)
template <typename T>
struct PatT {
    T fp, fx, fpT, fxT, fpX, fxX;
};
using Pat = PatT<double>;

// the pattern functions and their theta- and x-derivatives from the JKS
// coefficients a, b of one interferometer and P1, P2 = amp (cos 2psi, sin 2psi)
template <typename T>
__device__ __forceinline__ PatT<T> patterns_ab(T P1, T P2, T a, T b, T aT, T bT, T aX, T bX)
{
    PatT<T> p;
    p.fp = P1 * a + P2 * b;
    p.fx = P1 * b - P2 * a;
    p.fpT = P1 * aT + P2 * bT;
    p.fxT = P1 * bT - P2 * aT;
    p.fpX = P1 * aX + P2 * bX;
    p.fxX = P1 * bX - P2 * aX;
    return p;
}

template <typename T>
__device__ __forceinline__ PatT<T> patterns(T s2g, T c2g, T P1, T P2, const T (&J)[12])
{
    // J = a_s, a_c, b_c, b_s, then theta- and x-derivatives of each
    PatT<T> p;
    T a = s2g * J[0] + c2g * J[1], b = c2g * J[2] + s2g * J[3];
    T aT = s2g * J[4] + c2g * J[5], bT = c2g * J[6] + s2g * J[7];
    T aX = s2g * J[8] + c2g * J[9], bX = c2g * J[10] + s2g * J[11];
    p.fp = P1 * a + P2 * b;
    p.fx = P1 * b - P2 * a;
    p.fpT = P1 * aT + P2 * bT;
    p.fxT = P1 * bT - P2 * aT;
    p.fpX = P1 * aX + P2 * bX;
    p.fxX = P1 * bX - P2 * aX;
    return p;
}

// phase-derivative values common to all IFOs of one site at one point
template <typename T>
struct PhaseT {
    T Mc, eta, th, ph, tc, p9, p10;   // d Phi / d theta_i
    T tMc, teta;                      // Omega_E d tau*/d Mc, Omega_E d tau*/d eta
};
using Phase = PhaseT<double>;

// tangents of one IFO: real and imaginary parts
template <int NP, bool ROT, typename T>
__device__ __forceinline__ void tangents(const PatT<T> &p, T Acp, T Acx, T Adcp, T Adcx, T aMc,
                                         T invdL, const PhaseT<T> &ph, T (&gr)[NP], T (&gi)[NP],
                                         T &qr, T &qi)
{
    qr = Acp * p.fp;
    qi = Acx * p.fx;
    const T xr = Acp * p.fpX, xi = Acx * p.fxX;   // dQ/dx
    const T tr = Acp * p.fpT, ti = Acx * p.fxT;   // dQ/dtheta
    // Mc
    gr[0] = aMc * qr - qi * ph.Mc;
    gi[0] = aMc * qi + qr * ph.Mc;
    if (ROT) {
        gr[0] = fma(ph.tMc, xr, gr[0]);
        gi[0] = fma(ph.tMc, xi, gi[0]);
    }
    // eta
    gr[1] = -qi * ph.eta;
    gi[1] = qr * ph.eta;
    if (ROT) {
        gr[1] = fma(ph.teta, xr, gr[1]);
        gi[1] = fma(ph.teta, xi, gi[1]);
    }
    // dL
    gr[2] = -qr * invdL;
    gi[2] = -qi * invdL;
    // theta
    gr[3] = tr - qi * ph.th;
    gi[3] = ti + qr * ph.th;
    // phi (x = phi - lon - Omega_E t)
    gr[4] = xr - qi * ph.ph;
    gi[4] = xi + qr * ph.ph;
    // iota
    gr[5] = Adcp * p.fp;
    gi[5] = Adcx * p.fx;
    // psi: dF+/dpsi = 2 Fx, dFx/dpsi = -2 F+
    gr[6] = 2.0 * Acp * p.fx;
    gi[6] = -2.0 * Acx * p.fp;
    // tc: dx/dtc = -Omega_E
    gr[7] = -qi * ph.tc;
    gi[7] = qr * ph.tc;
    if (ROT) {
        gr[7] = fma(-OMEGA_E, xr, gr[7]);
        gi[7] = fma(-OMEGA_E, xi, gi[7]);
    }
    // Phic: dPhi/dPhic = -1
    gr[8] = qi;
    gi[8] = -qr;
    if (NP == 11) {
        gr[NP - 2] = -qi * ph.p9;
        gi[NP - 2] = qr * ph.p9;
        gr[NP - 1] = -qi * ph.p10;
        gi[NP - 1] = qr * ph.p10;
    }
}

// ln S_n at ln f for tabulated PSD p: the segment j with ln f_j <= ln f <=
// ln f_j+1, found by bisection the first time and then by walking forward (a
// lane's grid points increase); +inf (zero weight) outside the table
__device__ __forceinline__ double psd_table_lns(const DevNet &net, int p, double x, int &seg)
{
    const PsdSeg *T = net.psd_seg + net.psd_seg0[p];
    const int n = net.psd_nseg[p];
    if (isnan(__ldg(&T[0].lns))) return NAN;   // a table that breaks its rules
    if (!(x >= __ldg(&T[0].lnf)) || !(x <= __ldg(&T[n - 1].lnf1))) return INFINITY;
    if (seg < 0 || x < __ldg(&T[seg].lnf)) {
        int lo = 0, hi = n - 1;          // largest j with ln f_j <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&T[mid].lnf) <= x) lo = mid;
            else hi = mid - 1;
        }
        seg = lo;
    }
    while (seg < n - 1 && x > __ldg(&T[seg].lnf1)) seg++;
    return fma(__ldg(&T[seg].slope), x - __ldg(&T[seg].lnf), __ldg(&T[seg].lns));
}

// PN terms at one grid point v = (pi M f)^(1/3): the frequency, the phase
// derivatives d Psi/d Mc, d Psi/d eta (basis of 11 powers of v, ln v) and of
// slots 9, 10, and (rotation) tau*(f) with its Mc and eta derivatives
template <typename T>
struct PnTermsT {
    T f, vi3, dMc, dEt, d9, d10, tau, tMc, tEt;
};
using PnTerms = PnTermsT<double>;

template <int NP, bool ROT, typename T>
__device__ __forceinline__ PnTermsT<T> pn_terms(const T *E, T v, T vinv, T lnv)
{
    PnTermsT<T> t;
    const T vi2 = vinv * vinv, vi3 = vi2 * vinv, vi5 = vi3 * vi2;
    const T v2 = v * v, v5 = v2 * v2 * v, v7 = v5 * v2, vl = v * lnv;
    t.vi3 = vi3;
    t.f = v2 * v * E[EV_INV_PIM];
    const T *PM = E + EV_PM, *PE = E + EV_PE;
    if constexpr (std::is_same<T, dfl>::value) {
        // d Psi/d Mc and d Psi/d eta together on the packed FP32x2 instructions
        // (the Mc polynomial's ln v coefficient is zero: adding its term is exact)
        auto pr = [&](int q) { return d2_make(PM[q], PE[q]); };
        dfl2 d = pr(8) * d2_bcast(v7);
        d = pr(7) * d2_bcast(v5) + d;
        d = pr(10) * d2_bcast(vl) + d;
        d = pr(9) * d2_bcast(lnv) + d;
        d = pr(6) * d2_bcast(v2) + d;
        d = pr(5) * d2_bcast(v) + d;
        d = pr(4) + d;
        d = pr(3) * d2_bcast(vinv) + d;
        d = pr(2) * d2_bcast(vi2) + d;
        d = pr(1) * d2_bcast(vi3) + d;
        d = pr(0) * d2_bcast(vi5) + d;
        t.dMc = d2_x(d);
        t.dEt = d2_y(d);
        t.d9 = t.d10 = T(0.0);
        if (NP == 11) {
            const T *P9 = E + EV_P9, *P10 = E + EV_P10;
            auto p9 = [&](int q) { return d2_make(P9[q], P10[q]); };
            const dfl2 e = p9(0) * d2_bcast(vi2) +
                           (p9(1) * d2_bcast(vinv) + (p9(2) * d2_bcast(v5) + p9(3) * d2_bcast(v7)));
            t.d9 = d2_x(e);
            t.d10 = d2_y(e);
        }
    } else {
        T dMc = PM[8] * v7;
        dMc = fma(PM[7], v5, dMc);
        dMc = fma(PM[10], vl, dMc);
        dMc = fma(PM[6], v2, dMc);
        dMc = fma(PM[5], v, dMc);
        dMc = PM[4] + dMc;
        dMc = fma(PM[3], vinv, dMc);
        dMc = fma(PM[2], vi2, dMc);
        dMc = fma(PM[1], vi3, dMc);
        dMc = fma(PM[0], vi5, dMc);
        asm volatile("" ::: "memory");   // keep coefficient loads local (register pressure)
        T dEt = PE[8] * v7;
        dEt = fma(PE[7], v5, dEt);
        dEt = fma(PE[10], vl, dEt);
        dEt = fma(PE[9], lnv, dEt);
        dEt = fma(PE[6], v2, dEt);
        dEt = fma(PE[5], v, dEt);
        dEt = PE[4] + dEt;
        dEt = fma(PE[3], vinv, dEt);
        dEt = fma(PE[2], vi2, dEt);
        dEt = fma(PE[1], vi3, dEt);
        dEt = fma(PE[0], vi5, dEt);
        asm volatile("" ::: "memory");
        t.dMc = dMc;
        t.dEt = dEt;
        t.d9 = t.d10 = T(0.0);
        if (NP == 11) {
            const T *P9 = E + EV_P9, *P10 = E + EV_P10;
            t.d9 = fma(P9[0], vi2, fma(P9[1], vinv, fma(P9[2], v5, P9[3] * v7)));
            t.d10 = fma(P10[0], vi2, fma(P10[1], vinv, fma(P10[2], v5, P10[3] * v7)));
        }
    }
    // tau*(f) and its derivatives (rotation only)
    t.tau = t.tMc = t.tEt = T(0.0);
    if (ROT) {
        const T *T0 = E + EV_T0, *TM = E + EV_TM, *TE = E + EV_TE;
        const T b[8] = {vi5, vi3, vi2, vinv, T(1.0), v, v2, vl};
        T s0 = T0[7] * b[7];
#pragma unroll
        for (int q = 6; q >= 0; q--) s0 = fma(T0[q], b[q], s0);
        t.tau = s0 * vi3;
        if constexpr (std::is_same<T, dfl>::value) {
            // double-float pass: the Mc and eta derivatives of tau* in FP32.
            // They enter only the Earth-rotation parts of the Mc and eta
            // tangents, Omega_E dtau*/dtheta dQ/dx, about Omega_E / (2 pi f)
            // (< 1e-5) of those tangents, so an FP32 rounding there is ~1e-12
            // of the tangent, below the double-float arithmetic's own error
            // amplified through the Gram
            float s1 = TM[7].hi * b[7].hi, s2 = TE[7].hi * b[7].hi;
#pragma unroll
            for (int q = 6; q >= 0; q--) {
                s1 = fmaf(TM[q].hi, b[q].hi, s1);
                s2 = fmaf(TE[q].hi, b[q].hi, s2);
            }
            t.tMc = dfl(s1 * vi3.hi, 0.0f);
            t.tEt = dfl(s2 * vi3.hi, 0.0f);
        } else {
            T s1 = TM[7] * b[7], s2 = TE[7] * b[7];
#pragma unroll
            for (int q = 6; q >= 0; q--) {
                s1 = fma(TM[q], b[q], s1);
                s2 = fma(TE[q], b[q], s2);
            }
            t.tMc = s1 * vi3;
            t.tEt = s2 * vi3;
        }
        asm volatile("" ::: "memory");
    }
    return t;
}

// amplitude times the square root of the noise weight per PSD:
// sigma_p = A sqrt(W_p), W_p = 4 w / S_p(f) at grid point k of weight w
template <bool TAB>
__device__ __forceinline__ void psd_sigma(const DevNet &net, const double *E, int k, double f,
                                          double vi3, double w, double Aamp, int (&tseg)[MAX_PSD],
                                          double (&Wp)[MAX_PSD])
{
#pragma unroll
    for (int p = 0; p < MAX_PSD; p++) {
        if (TAB && p < net.n_psd && net.psd_kind[p] == 1) {
            // tabulated PSD: ln S on the log-log segment holding ln f
            // (blind outside the table: zero weight)
            const double lnf_k = fma((double)k, E[EV_LNR], E[EV_LNF0]);
            const double lns = psd_table_lns(net, p, lnf_k, tseg[p]);
            Wp[p] = Aamp * sqrt(4.0 * w) * exp(-0.5 * lns);
        } else if (p < net.n_psd) {
            const double x = f * net.psd_inv_f0[p];
            const double xi = net.psd_f0[p] * E[EV_PIM] * vi3;
            double S = 0.0;
            for (int q = 0; q < net.psd_nterm[p]; q++) {
                const int pw = net.psd_pow[p][q];
                S = fma(net.psd_coef[p][q], pw >= 0 ? ipow(x, pw) : ipow(xi, -pw), S);
            }
            Wp[p] = Aamp * sqrt(4.0 * w * rcp64(S));
        } else {
            Wp[p] = 0.0;
        }
    }
}

// site terms at one grid point: the pattern-function coefficients J at the
// Earth angle x = x0 + Omega_E tau* (rotation) and the phase derivatives,
// including the Doppler phase, shared by the site's interferometers
template <int MODE, bool ROT, typename T>
__device__ __forceinline__ void site_terms(const T *S, const PnTermsT<T> &pn, T twopif,
                                           T (&J)[12], PhaseT<T> &ph)
{
    const T x = ROT ? fma(T(OMEGA_E), pn.tau, S[SC_X0]) : S[SC_X0];
    T sx, cxx;
    sincos(x, &sx, &cxx);
    const T c2x = fma(T(2.0) * cxx, cxx, T(-1.0)), s2x = T(2.0) * sx * cxx;
    if constexpr (std::is_same<T, dfl>::value) {
        // the same operations, two coefficients at a time on the packed FP32x2
        // instructions (the pairs share their structure a u + b w [+ c])
        auto two = [](dfl a) { return dfl(2.0f * a.hi, 2.0f * a.lo); };   // exact
        const dfl2 sc2 = d2_make(s2x, c2x);
        const dfl2 cc = d2_bcast(c2x), ss = d2_bcast(s2x), cx = d2_bcast(cxx), sq = d2_bcast(sx);
        const dfl2 xc = d2_make(sx, cxx);
        dfl2 p;
        p = d2_make(S[SC_A1], S[SC_A1T]) * cc +
            (d2_make(S[SC_A2], S[SC_A2T]) * cx + d2_make(S[SC_A3], S[SC_A3T]));
        J[0] = d2_x(p), J[4] = d2_y(p);
        p = d2_make(S[SC_A4], S[SC_B1]) * sc2 + d2_make(S[SC_A5], S[SC_B2]) * xc;
        J[1] = d2_x(p), J[2] = d2_y(p);
        p = d2_make(S[SC_B3], S[SC_B1T]) * sc2 + d2_make(S[SC_B4], S[SC_B2T]) * xc;
        J[3] = d2_x(p), J[6] = d2_y(p);
        p = d2_make(S[SC_A4T], S[SC_B3T]) * ss + d2_make(S[SC_A5T], S[SC_B4T]) * sq;
        J[5] = d2_x(p), J[7] = d2_y(p);
        p = d2_make(-two(S[SC_A1]), two(S[SC_A4])) * sc2 + d2_make(-S[SC_A2], S[SC_A5]) * xc;
        J[8] = d2_x(p), J[9] = d2_y(p);
        p = d2_make(-two(S[SC_B1]), two(S[SC_B3])) * sc2 + d2_make(-S[SC_B2], S[SC_B4]) * xc;
        J[10] = d2_x(p), J[11] = d2_y(p);
    } else {
        J[0] = fma(S[SC_A1], c2x, fma(S[SC_A2], cxx, S[SC_A3]));
        J[1] = fma(S[SC_A4], s2x, S[SC_A5] * sx);
        J[2] = fma(S[SC_B1], c2x, S[SC_B2] * cxx);
        J[3] = fma(S[SC_B3], s2x, S[SC_B4] * sx);
        J[4] = fma(S[SC_A1T], c2x, fma(S[SC_A2T], cxx, S[SC_A3T]));
        J[5] = fma(S[SC_A4T], s2x, S[SC_A5T] * sx);
        J[6] = fma(S[SC_B1T], c2x, S[SC_B2T] * cxx);
        J[7] = fma(S[SC_B3T], s2x, S[SC_B4T] * sx);
        J[8] = fma(-2.0 * S[SC_A1], s2x, -S[SC_A2] * sx);
        J[9] = fma(2.0 * S[SC_A4], c2x, S[SC_A5] * cxx);
        J[10] = fma(-2.0 * S[SC_B1], s2x, -S[SC_B2] * sx);
        J[11] = fma(2.0 * S[SC_B3], c2x, S[SC_B4] * cxx);
    }
    const T dxPD = -twopif * S[SC_D1] * sx;
    ph.th = twopif * fma(S[SC_D1T], cxx, S[SC_D2T]);
    ph.ph = dxPD;
    ph.Mc = pn.dMc;
    ph.eta = pn.dEt;
    ph.tc = twopif;
    ph.p9 = pn.d9;
    ph.p10 = pn.d10;
    ph.tMc = T(0.0);
    ph.teta = T(0.0);
    if (ROT) {
        // dx/dMc = Omega_E dtau*/dMc, dx/deta likewise, dx/dtc = -Omega_E
        ph.tMc = T(OMEGA_E) * pn.tMc;
        ph.teta = T(OMEGA_E) * pn.tEt;
        ph.Mc = fma(dxPD, ph.tMc, pn.dMc);
        ph.eta = fma(dxPD, ph.teta, pn.dEt);
        ph.tc = fma(T(-OMEGA_E), dxPD, twopif);
    }
    if (MODE == MODE_SNRGRAD) {
        ph.Mc = ph.eta = ph.th = ph.ph = ph.tc = ph.p9 = ph.p10 = T(0.0);
    }
}

template <int MODE, int NP, bool ROT, bool TAB, int G>
__global__ void __launch_bounds__(128) k_points_fp64(PointArgs A)
{
    constexpr int GPW = 32 / G;   // work groups (items in flight) per warp
    constexpr int NACC = NAccOf<MODE, NP>::value;
    constexpr int RS = G + 1;
    extern __shared__ double red_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane % G;
    const unsigned gmask = ((1u << G) - 1u) << (gid * G);
    double *red = red_smem + (wib * GPW + gid) * (NACC * RS);
    // per-group copy of the item's event constants (read every point from
    // shared memory instead of being held in registers across the loop)
    double *cs = red_smem + 4 * GPW * NACC * RS + (wib * GPW + gid) * EVC;
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;
    const DevNet &net = A.net;
    // work count from device memory (no host readback), bounded by the capacity
    const int64_t n_total = A.item_off[A.n_ev];
    const int64_t n_items = n_total < A.n_items ? n_total : A.n_items;

    for (int64_t it = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW + gid;
         it < n_items; it += ngroups) {
        const int64_t e = find_event(A.item_off, A.n_ev, it);
        const int64_t j = it - A.item_off[e];
        const int64_t nj = A.item_off[e + 1] - A.item_off[e];
        const double *Eg = A.evc + e * (int64_t)EVC;
        for (int q = gl; q < EVC; q += G) cs[q] = Eg[q];
        __syncwarp(gmask);
        const double *E = cs;
        const int N = (int)E[EV_NPTS];
        const int kb = (int)((int64_t)N * j / nj), ke = (int)((int64_t)N * (j + 1) / nj);

        double acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; a++) acc[a] = 0.0;

        // covariance of the event (logdet mode), packed upper
        double Cv[MODE == MODE_LOGDET ? NP * (NP + 1) / 2 : 1];
        bool skip = false;
        if (MODE == MODE_LOGDET) {
#pragma unroll
            for (int q = 0; q < NP * (NP + 1) / 2; q++) Cv[q] = A.cov[(int64_t)q * A.n_ev + e];
            skip = !isfinite(Cv[0]);
        }

        int k = kb + gl;
        if (k < ke && !skip) {
            const double lnr = E[EV_LNR];
            const double lnf = fma((double)k, lnr, E[EV_LNF0]);
            double lnv = (lnf + E[EV_LNPIM]) * (1.0 / 3.0);
            double v = exp(lnv), vinv = exp(-lnv);
            double Aamp = E[EV_A0] * exp(-7.0 / 6.0 * lnf);
            const double rho = E[adv_slot<G>(0)], rhoi = E[adv_slot<G>(1)];
            const double dlnv = E[adv_slot<G>(2)], rA = E[adv_slot<G>(3)];
            const double wc0 = E[EV_WC0], wcm = E[EV_WCM], wcn = E[EV_WCN];
            const double cp = E[EV_CP], cx = E[EV_CX], dcp = E[EV_DCP], dcx = E[EV_DCX];
            const double c2p = E[EV_C2PSI], s2p = E[EV_S2PSI];
            const double aMc = E[EV_AMC], invdL = E[EV_INVDL];
            int tseg[MAX_PSD];   // current segment of each tabulated PSD (-1: not found yet)
#pragma unroll
            for (int p = 0; p < MAX_PSD; p++) tseg[p] = -1;

#pragma unroll 1
            for (; k < ke; k += G) {
                // ---- grid point, weight, PN terms
                const PnTerms pn = pn_terms<NP, ROT>(E, v, vinv, lnv);
                const double w = pn.f * (k == 0 ? wc0 : (k == N - 1 ? wcn : wcm));
                const double twopif = TWO_PI * pn.f;
                // ---- amplitude times sqrt of the noise weight per PSD:
                //      sigma = A sqrt(W), W = 4 w / S_n(f); tangents are scaled by it
                double Wp[MAX_PSD];
                psd_sigma<TAB>(net, E, k, pn.f, pn.vi3, w, Aamp, tseg, Wp);

                // ---- sites
#pragma unroll 1
                for (int s = 0; s < net.n_site; s++) {
                    // (site s is detector s) log-det gradient: only the requested detectors
                    if (MODE == MODE_LOGDET && !((A.det_mask >> s) & 1u)) continue;
                    const double *S = A.sitec + (e * net.n_site + s) * (int64_t)SC_N;
                    if (net.masked && S[SC_SLOT0] < 0.0) continue;   // every arm of the site off
                    double J[12];
                    Phase ph;
                    site_terms<MODE, ROT>(S, pn, twopif, J, ph);
#pragma unroll 1
                    for (int slot = 0; slot < net.site_nslot[s]; slot++) {
                        // interferometer of this slot; an empty slot (duty factor)
                        // runs with amplitude 0, so every group of a warp takes
                        // the same path
                        int q = net.masked ? (int)S[SC_SLOT0 + slot] : net.site_ifo0[s] + slot;
                        double on = 1.0;
                        if (q < 0) {
                            q = net.site_ifo0[s];
                            on = 0.0;
                        }
                        const double amp = net.ifo_amp[q] * on;
                        const Pat pt = patterns(net.ifo_s2g[q], net.ifo_c2g[q], amp * c2p,
                                                amp * s2p, J);
                        const double sg = Wp[net.ifo_psd[q]];
                        double gr[NP], gi[NP], qr, qi;
                        tangents<NP, ROT>(pt, sg * cp, sg * cx, sg * dcp, sg * dcx, aMc, invdL, ph,
                                          gr, gi, qr, qi);
                        const double q2 = fma(qr, qr, qi * qi);
                        if (MODE == MODE_FISHER) {
                            acc[0] += q2;
                            int a = 1;
#pragma unroll
                            for (int i = 0; i < NP; i++)
#pragma unroll
                                for (int jj = i; jj < NP; jj++) {
                                    acc[a] = fma(gr[i], gr[jj], fma(gi[i], gi[jj], acc[a]));
                                    a++;
                                }
                        } else if (MODE == MODE_SNR) {
                            acc[0] += q2;
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc[1 + d] += q2;
                        } else if (MODE == MODE_SNRGRAD) {
                            // Re(Q^* g_i) = Re(Q^* dQ/dtheta_i): the phase part i Q dPhi
                            // contributes exactly zero, so it is left out (it would only
                            // add rounding), and Phic / slots 9, 10 stay exactly 0.
                            acc[0] += q2;
#pragma unroll
                            for (int i = 0; i < 8; i++)
                                acc[1 + i] = fma(qr, gr[i], fma(qi, gi[i], acc[1 + i]));
                            // the detector's orientation: the patterns are linear in
                            // (sin 2 gamma, cos 2 gamma), so dQ/dgamma is Q with
                            // (sin 2 gamma, cos 2 gamma) -> (2 cos 2 gamma, -2 sin 2 gamma)
                            const Pat pg = patterns(2.0 * net.ifo_c2g[q], -2.0 * net.ifo_s2g[q],
                                                    amp * c2p, amp * s2p, J);
                            const double qgr = sg * cp * pg.fp, qgi = sg * cx * pg.fx;
                            const double rg = fma(qr, qgr, qi * qgi);
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc[1 + NP + d] += rg;
                        } else {   // MODE_LOGDET
                            // y = C g
                            double yr[NP], yi[NP];
#pragma unroll
                            for (int i = 0; i < NP; i++) {
                                double sr = 0.0, si = 0.0;
#pragma unroll
                                for (int m = 0; m < NP; m++) {
                                    const int lo = i < m ? i : m, hi = i < m ? m : i;
                                    const double c = Cv[lo * NP - lo * (lo - 1) / 2 + (hi - lo)];
                                    sr = fma(c, gr[m], sr);
                                    si = fma(c, gi[m], si);
                                }
                                yr[i] = sr;
                                yi[i] = si;
                            }
                            // g' = d g / d gamma: the same tangents with (sin2g, cos2g)
                            // replaced by (2 cos2g, -2 sin2g)
                            const Pat pd = patterns(2.0 * net.ifo_c2g[q], -2.0 * net.ifo_s2g[q],
                                                    amp * c2p, amp * s2p, J);
                            double hr[NP], hi_[NP], dqr, dqi;
                            tangents<NP, ROT>(pd, sg * cp, sg * cx, sg * dcp, sg * dcx, aMc, invdL,
                                              ph, hr, hi_, dqr, dqi);
                            double t = 0.0;
#pragma unroll
                            for (int i = 0; i < NP; i++) t = fma(hr[i], yr[i], fma(hi_[i], yi[i], t));
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc[d] = fma(2.0, t, acc[d]);
                        }
                    }
                }
                // ---- advance to the lane's next point (k + G)
                v *= rho;
                vinv *= rhoi;
                lnv += dlnv;
                Aamp *= rA;
            }
        }
        // ---- group reduction through shared memory, fixed order
#pragma unroll
        for (int a = 0; a < NACC; a++) red[a * RS + gl] = acc[a];
        __syncwarp(gmask);
        double *out = A.partial + it * (int64_t)A.nacc;
        for (int a = gl; a < A.nacc; a += G) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < G; l++) s += red[a * RS + l];
            out[a] = s;
        }
        __syncwarp(gmask);
    }
}

template <int MODE, int NP, bool ROT, bool TAB, int G>
cudaError_t launch_one(const PointArgs &a, cudaStream_t s)
{
    constexpr int NACC = NAccOf<MODE, NP>::value;
    constexpr int GPW = 32 / G;
    const size_t smem = ((size_t)4 * GPW * NACC * (G + 1) + (size_t)4 * GPW * EVC) * sizeof(double);
    static PerDeviceOnce attr;
    cudaError_t err = set_smem_once(attr, k_points_fp64<MODE, NP, ROT, TAB, G>, smem);
    if (err != cudaSuccess) return err;
    if (a.n_items <= 0) return cudaSuccess;
    k_points_fp64<MODE, NP, ROT, TAB, G><<<points_grid_size(a.blocks_per_sm), 128, smem, s>>>(a);
    return cudaGetLastError();
}

// the Fisher pass runs the tile the caller chose (lanes per work item G; the
// autotuner's choice), the other passes, and networks with a tabulated PSD, G = 8
template <int MODE, int NP, bool ROT, bool TAB>
cudaError_t launch_g(const PointArgs &a, cudaStream_t s)
{
    // (tabulated PSDs: G = 8 only, to bound the number of instantiations)
    if (MODE == MODE_FISHER && !TAB && a.group == 4) return launch_one<MODE, NP, ROT, TAB, 4>(a, s);
    if (MODE == MODE_FISHER && !TAB && a.group == 16) return launch_one<MODE, NP, ROT, TAB, 16>(a, s);
    return launch_one<MODE, NP, ROT, TAB, 8>(a, s);
}

template <int MODE, bool TAB>
cudaError_t launch_mode_t(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    if (np == 9)
        return rot ? launch_g<MODE, 9, true, TAB>(a, s) : launch_g<MODE, 9, false, TAB>(a, s);
    return rot ? launch_g<MODE, 11, true, TAB>(a, s) : launch_g<MODE, 11, false, TAB>(a, s);
}

// networks with a tabulated PSD run the instantiation that evaluates tables
template <int MODE>
cudaError_t launch_mode(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return has_psd_table(a.net) ? launch_mode_t<MODE, true>(np, rot, a, s)
                                : launch_mode_t<MODE, false>(np, rot, a, s);
}

}  // namespace

}  // namespace gw
