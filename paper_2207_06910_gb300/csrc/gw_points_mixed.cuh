// gw_points_mixed.cuh -- the fused point loop in mixed precision (kernel
// templates; instantiated by gw_points_mixed.cu and gw_points_mixed_fisher.cu).
//
// GB300 runs FP32 at ~58x its FP64 rate (FFMA 117 vs DFMA 2 per clock and SM),
// so this kernel keeps the FP64 pipe almost idle:
//  * high precision without FP64: the log grid (v = (pi M f)^(1/3), 1/v, ln v
//    by recurrence), the TaylorF2 phase derivatives d Psi/d theta_i, tau*(f)
//    and its derivatives, and the Earth angle x = x0 + Omega_E tau* are
//    evaluated in double-float arithmetic (value = hi + lo, two FP32 numbers,
//    ~2^-48 relative; error-free transforms of Knuth (two-sum) and Dekker
//    (product with an FMA)), then rounded once to FP32;
//  * FP32: noise weight, amplitude, pattern functions, Doppler derivatives,
//    tangents g_i and the products Re(g_i^* g_j);
//  * sums: every product is split exactly (p = a b, e = fma(a, b, -p)) and
//    added to a double-float accumulator with a two-sum, so Gamma_ij is the
//    exact sum of the FP32 products to ~1e-13 relative.  The rounding left is
//    that of each tangent once per point: it perturbs Gamma as a Gram matrix of
//    slightly perturbed vectors, not element by element.
// Tangents are pre-scaled by sigma = A sqrt(4 w / S_n), so the weight sits in
// the products; a rounding of sigma is a common factor of a point's tangents,
// i.e. a perturbation of the noise weight.
// FP64 is used only once per lane and work item (start of the recurrences)
// and in the final per-item sum.
#pragma once

#include <cmath>

#include "gw_dot2.cuh"
#include "gw_kernels.cuh"

namespace gw {

namespace {

// ---------------------------------------------------------------- double-float
// (the double-float type and the compensated dot products are in gw_dot2.cuh)
using DF = dfl;

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return DF{s, b - (s - a)};
}

__device__ __forceinline__ DF df_mul(DF x, DF y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_add(DF x, DF y)
{
    DF s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF df_of(float2 c) { return DF{c.x, c.y}; }

__device__ __forceinline__ DF df_from_double(double x)
{
    const float hi = (float)x;
    return DF{hi, (float)(x - (double)hi)};
}

// Compensated accumulation of the elementwise product a * b (two lanes: real
// and imaginary parts) into a packed double-float accumulator that holds the
// NEGATED sum: hn (register) + *ln (shared memory).  nb = -b.  q = fl(-a b) is
// added to hn with Knuth's two-sum s + t2 + t3 = hn + q, where t2 = hn's and
// t3 = q - bb q's roundoff (bb = s - hn).  The correction the sum needs is
// t2 + t3 - e with e = a b + q the product's exact rounding error; since
// t3 - e = -(a b + bb), it is t2 - fma(a, b, bb): one FMA replaces the product
// error and q's roundoff, and rounds only a quantity of roundoff size
// (|a b + bb| <= |e| + |t3|), so hn + ln = -(sum of a b) to ~2^-48 relative.
__device__ __forceinline__ void acc_pk(float2 &hn, float2 *ln, float2 a, float2 b, float2 nb)
{
    const float2 q = __fmul2_rn(a, nb);
    const float2 s = __fadd2_rn(hn, q);
    const float2 bb = f2sub(s, hn);
    const float2 t2 = f2sub(hn, f2sub(s, bb));
    const float2 y = __ffma2_rn(a, b, bb);
    hn = s;
    *ln = __fadd2_rn(*ln, f2sub(t2, y));
}

__device__ __forceinline__ int64_t find_event_m(const int64_t *off, int64_t n, int64_t it)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float ipowf(float x, int p)
{
    float r = 1.0f;
    while (p) {
        if (p & 1) r *= x;
        x *= x;
        p >>= 1;
    }
    return r;
}

template <int MODE, int NP>
struct NAccM {
    static constexpr int value = MODE == MODE_FISHER ? 1 + NP * (NP + 1) / 2 + N_SNRGRAD_X
                               : MODE == MODE_SNRGRAD ? 1 + NP + MAX_DET
                               : 1 + MAX_DET;
};

struct PatF {
    float fp, fx, fpT, fxT, fpX, fxX;
};

__device__ __forceinline__ PatF patterns_f(float s2g, float c2g, float P1, float P2,
                                           const float (&J)[12])
{
    PatF p;
    float a = s2g * J[0] + c2g * J[1], b = c2g * J[2] + s2g * J[3];
    float aT = s2g * J[4] + c2g * J[5], bT = c2g * J[6] + s2g * J[7];
    float aX = s2g * J[8] + c2g * J[9], bX = c2g * J[10] + s2g * J[11];
    p.fp = P1 * a + P2 * b;
    p.fx = P1 * b - P2 * a;
    p.fpT = P1 * aT + P2 * bT;
    p.fxT = P1 * bT - P2 * aT;
    p.fpX = P1 * aX + P2 * bX;
    p.fxX = P1 * bX - P2 * aX;
    return p;
}

struct PhaseF {
    float Mc, eta, th, ph, tc, p9, p10, tMc, teta;
};

template <int NP, bool ROT>
__device__ __forceinline__ void tangents_f(const PatF &p, float Acp, float Acx, float Adcp,
                                           float Adcx, float aMc, float invdL, const PhaseF &ph,
                                           float (&gr)[NP], float (&gi)[NP], float &qr, float &qi,
                                           float &xr, float &xi, float &tr, float &ti)
{
    const float omega = (float)OMEGA_E;
    qr = Acp * p.fp;
    qi = Acx * p.fx;
    xr = Acp * p.fpX;      // dQ/dx
    xi = Acx * p.fxX;
    tr = Acp * p.fpT;      // dQ/dtheta
    ti = Acx * p.fxT;
    gr[0] = aMc * qr - qi * ph.Mc;
    gi[0] = aMc * qi + qr * ph.Mc;
    if (ROT) {
        gr[0] = fmaf(ph.tMc, xr, gr[0]);
        gi[0] = fmaf(ph.tMc, xi, gi[0]);
    }
    gr[1] = -qi * ph.eta;
    gi[1] = qr * ph.eta;
    if (ROT) {
        gr[1] = fmaf(ph.teta, xr, gr[1]);
        gi[1] = fmaf(ph.teta, xi, gi[1]);
    }
    gr[2] = -qr * invdL;
    gi[2] = -qi * invdL;
    gr[3] = tr - qi * ph.th;
    gi[3] = ti + qr * ph.th;
    gr[4] = xr - qi * ph.ph;
    gi[4] = xi + qr * ph.ph;
    gr[5] = Adcp * p.fp;
    gi[5] = Adcx * p.fx;
    gr[6] = 2.0f * Acp * p.fx;
    gi[6] = -2.0f * Acx * p.fp;
    gr[7] = -qi * ph.tc;
    gi[7] = qr * ph.tc;
    if (ROT) {
        gr[7] = fmaf(-omega, xr, gr[7]);
        gi[7] = fmaf(-omega, xi, gi[7]);
    }
    gr[8] = qi;
    gi[8] = -qr;
    if (NP == 11) {
        gr[NP - 2] = -qi * ph.p9;
        gi[NP - 2] = qr * ph.p9;
        gr[NP - 1] = -qi * ph.p10;
        gi[NP - 1] = qr * ph.p10;
    }
}

// (ln S_n - ln scale_ref) at ln f = x (double-float) for tabulated PSD p, as a
// double-float: the log-log segment holding x, found by bisection the first
// time and then by walking forward (a lane's grid points increase); hi = +inf
// (zero weight) outside the table, NaN for a table that breaks its rules
__device__ __forceinline__ bool df_lt(DF a, float ah, float al)
{
    return a.hi < ah || (a.hi == ah && a.lo < al);
}

__device__ __forceinline__ DF psd_table_lns_df(const DevNet &net, int p, DF x, int &seg)
{
    const float4 *T = net.psd_seg_f + 2 * net.psd_seg0[p];
    const int n = net.psd_nseg[p];
    const float4 t0 = __ldg(&T[0]);
    if (isnan(t0.z)) return DF{NAN, 0.0f};
    const float4 tl = __ldg(&T[2 * (n - 1) + 1]);
    if (df_lt(x, t0.x, t0.y) || (x.hi > tl.y || (x.hi == tl.y && x.lo > tl.z)))
        return DF{INFINITY, 0.0f};
    if (seg < 0 || df_lt(x, __ldg(&T[2 * seg].x), __ldg(&T[2 * seg].y))) {
        int lo = 0, hi = n - 1;          // largest j with ln f_j <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const float4 tm = __ldg(&T[2 * mid]);
            if (!df_lt(x, tm.x, tm.y)) lo = mid;
            else hi = mid - 1;
        }
        seg = lo;
    }
    for (;;) {
        if (seg >= n - 1) break;
        const float4 tb = __ldg(&T[2 * seg + 1]);
        if (!(x.hi > tb.y || (x.hi == tb.y && x.lo > tb.z))) break;
        seg++;
    }
    const float4 a = __ldg(&T[2 * seg]), b = __ldg(&T[2 * seg + 1]);
    const DF dx = df_add(x, DF{-a.x, -a.y});
    const DF y = two_sum(a.z, b.x * df_round(dx));
    return DF{y.hi, y.lo + a.w};
}

template <int MODE, int NP, bool ROT, bool TAB, int G>
__global__ void __launch_bounds__(128, 2) k_points_mixed(PointArgs A)
{
    constexpr int GPW = 32 / G;   // work groups (items in flight) per warp
    constexpr int NACC = NAccM<MODE, NP>::value;
    constexpr int NT = 128;         // threads per block
    extern __shared__ float red_f[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane % G;
    const unsigned gmask = ((1u << G) - 1u) << (gid * G);
    // compensation terms of the packed accumulators: lo[a * LDS + thread]
    // (row stride LDS = NT + 1 keeps the group reduction free of bank conflicts)
    constexpr int LDS = NT + 1;
    float2 *const lo_base = reinterpret_cast<float2 *>(red_f);
    float2 *mylo = lo_base + threadIdx.x;
    // per-group copy of the item's polynomial coefficients (slots EV_PM ..
    // EVC - 1, read every point from shared memory instead of being held in
    // registers across the loop)
    float2 *cs = lo_base + ((NACC * LDS + 1) & ~1) + (wib * GPW + gid) * NCOEF;
    // per-group copy of the item's scalar constants EV_WC0 .. EV_INVDL, read
    // where they are used (held in registers they would crowd out the sums)
    float2 *csc = lo_base + ((NACC * LDS + 1) & ~1) + 4 * GPW * NCOEF +
                  (wib * GPW + gid) * NSCAL;
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GPW;
    const DevNet &net = A.net;
    // work count from device memory (no host readback), bounded by the capacity
    const int64_t n_total = A.item_off[A.n_ev];
    const int64_t n_items = n_total < A.n_items ? n_total : A.n_items;
    const DF two_pi = DF{6.28318548f, -1.74845553e-7f};          // 2 pi = hi + lo
    const DF omega_e = df_from_double(OMEGA_E);

    for (int64_t it = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GPW + gid;
         it < n_items; it += ngroups) {
        const int64_t e = find_event_m(A.item_off, A.n_ev, it);
        const int64_t j = it - A.item_off[e];
        const int64_t nj = A.item_off[e + 1] - A.item_off[e];
        const double *E = A.evc + e * (int64_t)EVC;
        const float2 *Eg = A.evc_f + e * (int64_t)EVC;
        {
            float *csf = reinterpret_cast<float *>(cs);
            for (int q = gl; q < NCOEF; q += G) {
                const float2 c = Eg[EV_PM + q];
                csf[coef_pos(q, 0)] = c.x;
                csf[coef_pos(q, 1)] = c.y;
            }
        }
        for (int q = gl; q < NSCAL; q += G) csc[q] = Eg[EV_WC0 + q];
        __syncwarp(gmask);
        const float *cf = reinterpret_cast<const float *>(cs);

        const int N = (int)E[EV_NPTS];
        const int kb = (int)((int64_t)N * j / nj), ke = (int)((int64_t)N * (j + 1) / nj);

        // accumulators: negated (real-part sum, imaginary-part sum) per entry
        float2 acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; a++) {
            acc[a] = make_float2(0.0f, 0.0f);
            mylo[a * LDS] = make_float2(0.0f, 0.0f);
        }

        int k = kb + gl;
        if (k < ke) {
            // start of the lane's recurrences (FP64, once per lane and item)
            const double lnf = fma((double)k, E[EV_LNR], E[EV_LNF0]);
            const double lnv_d = (lnf + E[EV_LNPIM]) * (1.0 / 3.0);
            DF v = df_from_double(exp(lnv_d));
            DF vinv = df_from_double(exp(-lnv_d));
            DF lnv = df_from_double(lnv_d);
            // amplitude A0 f^(-7/6) as a double-float recurrence (an FP32 one
            // would drift by ~1e-6 over a lane's points)
            DF Aamp = df_from_double(E[EV_A0] * net.inv_sqrt_scale_ref * exp(-7.0 / 6.0 * lnf));
            // recurrence factors over G points (the G = 8 ones are in the scalar copy)
            const DF rhoG = G == 8 ? df_of(csc[EV_RHOG - EV_WC0]) : df_of(Eg[adv_slot<G>(0)]);
            const DF rhoiG = G == 8 ? df_of(csc[EV_RHOIG - EV_WC0]) : df_of(Eg[adv_slot<G>(1)]);
            const DF lnrhoG = G == 8 ? df_of(csc[EV_LNRHOG - EV_WC0]) : df_of(Eg[adv_slot<G>(2)]);
            const DF raG = G == 8 ? df_of(csc[EV_RAG - EV_WC0]) : df_of(Eg[adv_slot<G>(3)]);
            int tseg[MAX_PSD];   // current segment of each tabulated PSD (-1: not found yet)
#pragma unroll
            for (int p = 0; p < MAX_PSD; p++) tseg[p] = -1;
#define SC(slot) csc[(slot) - EV_WC0]

#pragma unroll 1
            for (; k < ke; k += G) {
                // ---------------- double-float part
                const DF vi2 = df_mul(vinv, vinv), vi3 = df_mul(vi2, vinv);
                const DF vi5 = df_mul(vi3, vi2);
                const DF v2 = df_mul(v, v), v3 = df_mul(v2, v), v5 = df_mul(v3, v2);
                const DF v7 = df_mul(v5, v2), vl = df_mul(v, lnv);
                const DF one = DF{1.0f, 0.0f};
                const DF b11[11] = {vi5, vi3, vi2, vinv, one, v, v2, v5, v7, lnv, vl};
                const float nb11[11] = {-vi5.hi, -vi3.hi, -vi2.hi, -vinv.hi, -1.0f, -v.hi,
                                        -v2.hi, -v5.hi, -v7.hi, -lnv.hi, -vl.hi};
                // (the empty asm statements keep the compiler from loading every
                // coefficient of every polynomial at once, which spills registers)
                const DF2 pmpe = dot2_pk<11>(reinterpret_cast<const float4 *>(cf + CO_PMPE), b11, nb11);
                const float dMcf = pmpe.hi.x + pmpe.lo.x;
                const float dEtf = pmpe.hi.y + pmpe.lo.y;
                asm volatile("" ::: "memory");
                float d9 = 0.0f, d10 = 0.0f;
                if (NP == 11) {
                    const DF b4[4] = {vi2, vinv, v5, v7};
                    const float nb4[4] = {-vi2.hi, -vinv.hi, -v5.hi, -v7.hi};
                    const DF2 p910 = dot2_pk<4>(reinterpret_cast<const float4 *>(cf + CO_P910), b4, nb4);
                    d9 = p910.hi.x + p910.lo.x;
                    d10 = p910.hi.y + p910.lo.y;
                    asm volatile("" ::: "memory");
                }
                DF tau = DF{0.0f, 0.0f};
                float tMc = 0.0f, tEt = 0.0f;
                if (ROT) {
                    const DF b8[8] = {vi5, vi3, vi2, vinv, one, v, v2, vl};
                    const float nb8[8] = {-vi5.hi, -vi3.hi, -vi2.hi, -vinv.hi, -1.0f, -v.hi,
                                          -v2.hi, -vl.hi};
                    tau = df_mul(dot2_s<8>(reinterpret_cast<const float2 *>(cf + CO_T0), b8), vi3);
                    asm volatile("" ::: "memory");
                    const DF2 tmte = dot2_pk<8>(reinterpret_cast<const float4 *>(cf + CO_TMTE), b8, nb8);
                    const float vi3f = df_round(vi3) * (float)OMEGA_E;
                    tMc = (tmte.hi.x + tmte.lo.x) * vi3f;
                    tEt = (tmte.hi.y + tmte.lo.y) * vi3f;
                    asm volatile("" ::: "memory");
                }
                const DF fdf = df_mul(v3, df_of(SC(EV_INV_PIM)));
                const float ff = df_round(fdf);
                const float twopif = (float)TWO_PI * ff;

                // ---------------- FP32: noise weight and amplitude per PSD
                const float w = ff * (k == 0 ? SC(EV_WC0).x : (k == N - 1 ? SC(EV_WCN).x : SC(EV_WCM).x));
                const float Af = df_round(Aamp);
                float sig[MAX_PSD];
#pragma unroll
                for (int p = 0; p < MAX_PSD; p++) {
                    if (TAB && p < net.n_psd && net.psd_kind[p] == 1) {
                        // tabulated PSD: 4 w / S = 4 w exp(-(ln S - ln S_ref)) relative to
                        // the reference scale, the exponent as a double-float (S itself
                        // would leave the FP32 range)
                        const DF lnf_df = df_add(df_mul(DF{3.0f, 0.0f}, lnv),
                                                 DF{-SC(EV_LNPIM).x, -SC(EV_LNPIM).y});
                        const DF y = psd_table_lns_df(net, p, lnf_df, tseg[p]);
                        sig[p] = Af * sqrtf(4.0f * w) * (expf(-0.5f * y.hi) * (1.0f - 0.5f * y.lo));
                    } else if (p < net.n_psd) {
                        const float x = ff * net.psd_inv_f0_f[p];
                        const float xi = 1.0f / x;
                        float S = 0.0f;
                        for (int q = 0; q < net.psd_nterm[p]; q++) {
                            const int pw = net.psd_pow[p][q];
                            S = fmaf(net.psd_coef_f[p][q], pw >= 0 ? ipowf(x, pw) : ipowf(xi, -pw), S);
                        }
                        sig[p] = Af * sqrtf(4.0f * w / S);
                    } else {
                        sig[p] = 0.0f;
                    }
                }

#pragma unroll 1
                for (int s = 0; s < net.n_site; s++) {
                    const float *S = A.sitec_f + (e * net.n_site + s) * (int64_t)SC_N;
                    if (net.masked && S[SC_SLOT0] < 0.0f) continue;  // every arm of the site off
                    float xs;
                    if (ROT) {
                        // x = x0 + Omega_E tau* in double-float, reduced to about [-pi, pi]
                        DF x = df_add(DF{S[SC_X0], S[SC_X0LO]}, df_mul(omega_e, tau));
                        const float kq = rintf(x.hi * 0.159154943f);
                        x = df_add(x, df_mul(two_pi, DF{-kq, 0.0f}));
                        xs = df_round(x);
                    } else {
                        xs = S[SC_X0];
                    }
                    float sx, cxx;
                    sincosf(xs, &sx, &cxx);
                    const float c2x = fmaf(2.0f * cxx, cxx, -1.0f), s2x = 2.0f * sx * cxx;
                    float J[12];
                    J[0] = fmaf(S[SC_A1], c2x, fmaf(S[SC_A2], cxx, S[SC_A3]));
                    J[1] = fmaf(S[SC_A4], s2x, S[SC_A5] * sx);
                    J[2] = fmaf(S[SC_B1], c2x, S[SC_B2] * cxx);
                    J[3] = fmaf(S[SC_B3], s2x, S[SC_B4] * sx);
                    J[4] = fmaf(S[SC_A1T], c2x, fmaf(S[SC_A2T], cxx, S[SC_A3T]));
                    J[5] = fmaf(S[SC_A4T], s2x, S[SC_A5T] * sx);
                    J[6] = fmaf(S[SC_B1T], c2x, S[SC_B2T] * cxx);
                    J[7] = fmaf(S[SC_B3T], s2x, S[SC_B4T] * sx);
                    J[8] = fmaf(-2.0f * S[SC_A1], s2x, -S[SC_A2] * sx);
                    J[9] = fmaf(2.0f * S[SC_A4], c2x, S[SC_A5] * cxx);
                    J[10] = fmaf(-2.0f * S[SC_B1], s2x, -S[SC_B2] * sx);
                    J[11] = fmaf(2.0f * S[SC_B3], c2x, S[SC_B4] * cxx);
                    PhaseF ph;
                    const float dxPD = -twopif * S[SC_D1] * sx;
                    ph.th = twopif * fmaf(S[SC_D1T], cxx, S[SC_D2T]);
                    ph.ph = dxPD;
                    ph.Mc = dMcf;
                    ph.eta = dEtf;
                    ph.tc = twopif;
                    ph.p9 = d9;
                    ph.p10 = d10;
                    ph.tMc = tMc;
                    ph.teta = tEt;
                    if (ROT) {
                        ph.Mc = fmaf(dxPD, tMc, dMcf);
                        ph.eta = fmaf(dxPD, tEt, dEtf);
                        ph.tc = fmaf(-(float)OMEGA_E, dxPD, twopif);
                    }
                    if (MODE == MODE_SNRGRAD) {
                        // Re(Q^* i Q dPhi) = 0: phase parts left out of the SNR gradient
                        ph.Mc = ph.eta = ph.th = ph.ph = ph.tc = ph.p9 = ph.p10 = 0.0f;
                    }
#pragma unroll 1
                    for (int slot = 0; slot < net.site_nslot[s]; slot++) {
                        // interferometer of this slot; an empty slot (duty factor)
                        // runs with amplitude 0, so every group of a warp takes
                        // the same path
                        int q = net.masked ? (int)S[SC_SLOT0 + slot] : net.site_ifo0[s] + slot;
                        float on = 1.0f;
                        if (q < 0) {
                            q = net.site_ifo0[s];
                            on = 0.0f;
                        }
                        const float amp = (float)net.ifo_amp[q] * on;
                        const PatF pt = patterns_f((float)net.ifo_s2g[q], (float)net.ifo_c2g[q],
                                                   amp * SC(EV_C2PSI).x, amp * SC(EV_S2PSI).x, J);
                        const float sg = sig[net.ifo_psd[q]];
                        float gr[NP], gi[NP], qr, qi, xr, xi, tr, ti;
                        tangents_f<NP, ROT>(pt, sg * SC(EV_CP).x, sg * SC(EV_CX).x, sg * SC(EV_DCP).x,
                                            sg * SC(EV_DCX).x, SC(EV_AMC).x, SC(EV_INVDL).x,
                                            ph, gr, gi, qr, qi, xr, xi, tr, ti);
                        // tangents as (real, imaginary) pairs
                        float2 Gt[NP];
#pragma unroll
                        for (int i = 0; i < NP; i++) Gt[i] = make_float2(gr[i], gi[i]);
                        const float2 Q = make_float2(qr, qi);
                        if (MODE == MODE_FISHER) {
                            // Gamma_ij: real and imaginary products summed separately
                            // (|Q|^2 = the (Phic, Phic) entry, copied at the end); the
                            // row's tangent is negated once for the whole row.  The d_L
                            // tangent is taken exactly as -Q/d_L: its row sums
                            // Re(g_j Q^*) and the reduction scales them by -1/d_L;
                            // (d_L, d_L) and (d_L, Phic) follow from (Phic, Phic) and
                            // Re(Q (iQ)^*) = 0, so they are not summed.
                            Gt[2] = Q;
                            int a = 1;
#pragma unroll
                            for (int i = 0; i < NP; i++) {
                                const float2 NGi = make_float2(-Gt[i].x, -Gt[i].y);
#pragma unroll
                                for (int jj = i; jj < NP; jj++) {
                                    if (!(i == 2 && (jj == 2 || jj == 8)))
                                        acc_pk(acc[a], mylo + a * LDS, Gt[jj], Gt[i], NGi);
                                    a++;
                                }
                                if (i & 1) asm volatile("" ::: "memory");
                            }
                            // phase-free SNR-gradient sums (see N_SNRGRAD_X)
                            constexpr int X0 = 1 + NP * (NP + 1) / 2;
                            const float2 X = make_float2(xr, xi), NX = make_float2(-xr, -xi);
                            const float2 T = make_float2(tr, ti);
                            const float2 NQ = make_float2(-qr, -qi);
                            acc_pk(acc[X0 + 0], mylo + (X0 + 0) * LDS, Q, X, NX);
                            acc_pk(acc[X0 + 1], mylo + (X0 + 1) * LDS,
                                   make_float2(ph.tMc * qr, ph.tMc * qi), X, NX);
                            acc_pk(acc[X0 + 2], mylo + (X0 + 2) * LDS,
                                   make_float2(ph.teta * qr, ph.teta * qi), X, NX);
                            acc_pk(acc[X0 + 3], mylo + (X0 + 3) * LDS, T, Q, NQ);
                            // X0 + 4, X0 + 5 (iota, psi) are the (iota, d_L), (psi, d_L)
                            // sums above
                        } else if (MODE == MODE_SNR) {
                            const float2 NQ = make_float2(-qr, -qi);
                            acc_pk(acc[0], mylo, Q, Q, NQ);
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc_pk(acc[1 + d], mylo + (1 + d) * LDS, Q, Q, NQ);
                        } else {   // MODE_SNRGRAD
                            const float2 NQ = make_float2(-qr, -qi);
                            acc_pk(acc[0], mylo, Q, Q, NQ);
#pragma unroll
                            for (int i = 0; i < 8; i++)
                                acc_pk(acc[1 + i], mylo + (1 + i) * LDS, Gt[i], Q, NQ);
                            // the detector's orientation: dQ/dgamma is Q with
                            // (sin 2 gamma, cos 2 gamma) -> (2 cos 2 gamma, -2 sin 2 gamma)
                            const PatF pg = patterns_f(2.0f * (float)net.ifo_c2g[q],
                                                       -2.0f * (float)net.ifo_s2g[q],
                                                       amp * SC(EV_C2PSI).x, amp * SC(EV_S2PSI).x, J);
                            const float2 QG = make_float2(sg * SC(EV_CP).x * pg.fp,
                                                          sg * SC(EV_CX).x * pg.fx);
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc_pk(acc[1 + NP + d], mylo + (1 + NP + d) * LDS, QG, Q, NQ);
                        }
                    }
                }
                v = df_mul(v, rhoG);
                vinv = df_mul(vinv, rhoiG);
                lnv = df_add(lnv, lnrhoG);
                Aamp = df_mul(Aamp, raG);
#undef SC
            }
        }
        // ---- group reduction.  Every lane collapses its (real, imaginary)
        // accumulators into one double-float value -(hn.x + hn.y + ln.x + ln.y)
        // and stores it over its compensation slot; then lane gl sums the
        // G lanes' values of the entries a = gl (mod G) in a fixed
        // order (error-free two-sum of the high parts, compensations added)
        // and writes them in FP64.
        // In the Fisher layout, slots whose value is another slot's sum are
        // filled first, from their source: SNR^2 and (d_L, d_L) from (Phic,
        // Phic) (scaled by 1/d_L^2 below), the iota and psi SNR-gradient sums
        // from the (d_L, iota) and (d_L, psi) sums; (d_L, Phic) stays zero.
        double *out = A.partial + it * (int64_t)A.nacc;
        constexpr int k88 = 1 + 8 * NP - 8 * 7 / 2, k22 = 1 + 2 * NP - 1;
        constexpr int X0 = 1 + NP * (NP + 1) / 2;
        auto collapse = [&](const int src, const int dst) {
            const float2 l2 = mylo[src * LDS];
            const DF h = two_sum(acc[src].x, acc[src].y);
            mylo[dst * LDS] = make_float2(-h.hi, -((l2.x + l2.y) + h.lo));
        };
        if (MODE == MODE_FISHER) {
            collapse(k88, 0);
            collapse(k88, k22);
            collapse(k22 + 3, X0 + 4);      // (d_L, iota)
            collapse(k22 + 4, X0 + 5);      // (d_L, psi)
        }
#pragma unroll
        for (int a = 0; a < NACC; a++)
            if (!(MODE == MODE_FISHER && (a == 0 || a == k22 || a == X0 + 4 || a == X0 + 5)))
                collapse(a, a);
        __syncwarp(gmask);
        const float2 *grp = lo_base + (threadIdx.x - gl);
#pragma unroll 1
        for (int a = gl; a < NACC; a += G) {
            const float2 *r = grp + a * LDS;
            float2 v0 = r[0];
            DF t = DF{v0.x, v0.y};
#pragma unroll
            for (int l = 1; l < G; l++) {
                const float2 u = r[l];
                const DF h = two_sum(t.hi, u.x);
                t = DF{h.hi, (t.lo + u.y) + h.lo};
            }
            double v = (double)t.hi + (double)t.lo + 0.0;
            if (MODE == MODE_FISHER) {
                // the d_L row sums Re(g_j Q^*): Gamma_{j,d_L} = -sum / d_L
                const double idl = A.evc[e * (int64_t)EVC + EV_INVDL];
                if (a == k22) v *= idl * idl;
                else if (a == 3 || a == NP + 2 || (a > k22 && a <= k22 + NP - 3)) v *= -idl;
            }
            if (a < A.nacc) out[a] = v;
        }
        __syncwarp(gmask);
    }
}

template <int MODE, int NP, bool ROT, bool TAB, int G>
cudaError_t launch_one_m(const PointArgs &a, cudaStream_t s)
{
    constexpr int NACC = NAccM<MODE, NP>::value;
    constexpr int GPW = 32 / G;
    const size_t smem = ((size_t)((NACC * 129 + 1) & ~1) + (size_t)4 * GPW * (NCOEF + NSCAL)) * sizeof(float2);
    static PerDeviceOnce attr;
    cudaError_t err = set_smem_once(attr, k_points_mixed<MODE, NP, ROT, TAB, G>, smem);
    if (err != cudaSuccess) return err;
    if (a.n_items <= 0) return cudaSuccess;
    k_points_mixed<MODE, NP, ROT, TAB, G><<<points_grid_size(a.blocks_per_sm), 128, smem, s>>>(a);
    return cudaGetLastError();
}

// the Fisher pass runs the tile the caller chose (lanes per work item G; the
// autotuner's choice), the other passes, and networks with a tabulated PSD, G = 8
template <int MODE, int NP, bool ROT, bool TAB>
cudaError_t launch_g_m(const PointArgs &a, cudaStream_t s)
{
    // (tabulated PSDs: G = 8 only, to bound the number of instantiations)
    if (MODE == MODE_FISHER && !TAB && a.group == 4) return launch_one_m<MODE, NP, ROT, TAB, 4>(a, s);
    if (MODE == MODE_FISHER && !TAB && a.group == 16) return launch_one_m<MODE, NP, ROT, TAB, 16>(a, s);
    return launch_one_m<MODE, NP, ROT, TAB, 8>(a, s);
}

template <int MODE, bool TAB>
cudaError_t launch_mode_mt(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    if (np == 9)
        return rot ? launch_g_m<MODE, 9, true, TAB>(a, s) : launch_g_m<MODE, 9, false, TAB>(a, s);
    return rot ? launch_g_m<MODE, 11, true, TAB>(a, s) : launch_g_m<MODE, 11, false, TAB>(a, s);
}

// networks with a tabulated PSD run the instantiation that evaluates tables
template <int MODE>
cudaError_t launch_mode_m(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    return has_psd_table(a.net) ? launch_mode_mt<MODE, true>(np, rot, a, s)
                                : launch_mode_mt<MODE, false>(np, rot, a, s);
}

}  // namespace

}  // namespace gw
