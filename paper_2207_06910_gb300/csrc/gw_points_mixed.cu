// gw_points_mixed.cu -- the fused point loop in mixed precision.
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
#include <cmath>

#include "gw_kernels.cuh"

namespace gw {

namespace {

// ---------------------------------------------------------------- double-float
struct DF {
    float hi, lo;
};

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

__device__ __forceinline__ float df_round(DF x) { return x.hi + x.lo; }

// sum_q c[q] b[q] in double-float
template <int N>
__device__ __forceinline__ DF df_dot(const float2 *c, const DF (&b)[N])
{
    DF s = df_mul(df_of(c[N - 1]), b[N - 1]);
#pragma unroll
    for (int q = N - 2; q >= 0; q--) s = df_add(s, df_mul(df_of(c[q]), b[q]));
    return s;
}

// packed FP32x2 subtraction (sm_100+)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}

// Exact accumulation of the elementwise product a * b (two lanes: real and
// imaginary parts) into a packed double-float accumulator that holds the
// NEGATED sum: hn (register) + *ln (shared memory).  nb = -b.  With p = fl(a b)
// and q = fl(a nb) = -p, e = fma(a, b, q) is the exact error of p; the two-sum
// of hn + q is exact; so hn + ln = -(sum of a b) up to the FP32 rounding of ln.
__device__ __forceinline__ void acc_pk(float2 &hn, float2 *ln, float2 a, float2 b, float2 nb)
{
    const float2 q = __fmul2_rn(a, nb);
    const float2 e = __ffma2_rn(a, b, q);
    const float2 s = __fadd2_rn(hn, q);
    const float2 bb = f2sub(s, hn);
    const float2 tn = __fadd2_rn(f2sub(hn, f2sub(s, bb)), f2sub(q, bb));
    hn = s;
    *ln = __fadd2_rn(*ln, f2sub(tn, e));
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
                               : MODE == MODE_SNRGRAD ? 1 + NP
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

template <int MODE, int NP, bool ROT>
__global__ void __launch_bounds__(128, 2) k_points_mixed(PointArgs A)
{
    constexpr int NACC = NAccM<MODE, NP>::value;
    constexpr int NT = 128;         // threads per block
    extern __shared__ float red_f[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gid = lane / GROUP, gl = lane % GROUP;
    const unsigned gmask = ((1u << GROUP) - 1u) << (gid * GROUP);
    // compensation terms of the packed accumulators: lo[a * NT + thread]
    float2 *mylo = reinterpret_cast<float2 *>(red_f) + threadIdx.x;
    // per-group copy of the item's event constants (read every point from
    // shared memory instead of being held in registers across the loop)
    float2 *cs = reinterpret_cast<float2 *>(red_f) + NACC * NT + (wib * GROUPS_PER_WARP + gid) * EVC;
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x >> 5) * GROUPS_PER_WARP;
    const DevNet &net = A.net;
    // work count from device memory (no host readback), bounded by the capacity
    const int64_t n_total = A.item_off[A.n_ev];
    const int64_t n_items = n_total < A.n_items ? n_total : A.n_items;
    const DF two_pi = DF{6.28318548f, -1.74845553e-7f};          // 2 pi = hi + lo
    const DF omega_e = df_from_double(OMEGA_E);

    for (int64_t it = ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * GROUPS_PER_WARP + gid;
         it < n_items; it += ngroups) {
        const int64_t e = find_event_m(A.item_off, A.n_ev, it);
        const int64_t j = it - A.item_off[e];
        const int64_t nj = A.item_off[e + 1] - A.item_off[e];
        const double *E = A.evc + e * (int64_t)EVC;
        const float2 *Eg = A.evc_f + e * (int64_t)EVC;
        for (int q = gl; q < EVC; q += GROUP) cs[q] = Eg[q];
        __syncwarp(gmask);
        const float2 *Ef = cs;
        const int N = (int)E[EV_NPTS];
        const int kb = (int)((int64_t)N * j / nj), ke = (int)((int64_t)N * (j + 1) / nj);

        // accumulators: negated (real-part sum, imaginary-part sum) per entry
        float2 acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; a++) {
            acc[a] = make_float2(0.0f, 0.0f);
            mylo[a * NT] = make_float2(0.0f, 0.0f);
        }

        int k = kb + gl;
        if (k < ke) {
            // start of the lane's recurrences (FP64, once per lane and item)
            const double lnf = fma((double)k, E[EV_LNR], E[EV_LNF0]);
            const double lnv_d = (lnf + E[EV_LNPIM]) * (1.0 / 3.0);
            DF v = df_from_double(exp(lnv_d));
            DF vinv = df_from_double(exp(-lnv_d));
            DF lnv = df_from_double(lnv_d);
            float Aamp = (float)(E[EV_A0] * net.inv_sqrt_scale_ref) *
                         expf((float)(-7.0 / 6.0 * lnf));
            const DF rho = df_of(Ef[EV_RHOG]), rhoi = df_of(Ef[EV_RHOIG]);
            const DF dlnv = df_of(Ef[EV_LNRHOG]);
            const DF inv_pim = df_of(Ef[EV_INV_PIM]);
            const float rA = Ef[EV_RAG].x;
            const float wc0 = Ef[EV_WC0].x, wcm = Ef[EV_WCM].x, wcn = Ef[EV_WCN].x;
            const float cp = Ef[EV_CP].x, cx = Ef[EV_CX].x;
            const float dcp = Ef[EV_DCP].x, dcx = Ef[EV_DCX].x;
            const float c2p = Ef[EV_C2PSI].x, s2p = Ef[EV_S2PSI].x;
            const float aMc = Ef[EV_AMC].x, invdL = Ef[EV_INVDL].x;

#pragma unroll 1
            for (; k < ke; k += GROUP) {
                // ---------------- double-float part
                const DF vi2 = df_mul(vinv, vinv), vi3 = df_mul(vi2, vinv);
                const DF vi5 = df_mul(vi3, vi2);
                const DF v2 = df_mul(v, v), v3 = df_mul(v2, v), v5 = df_mul(v3, v2);
                const DF v7 = df_mul(v5, v2), vl = df_mul(v, lnv);
                const DF one = DF{1.0f, 0.0f};
                const DF b11[11] = {vi5, vi3, vi2, vinv, one, v, v2, v5, v7, lnv, vl};
                // (the empty asm statements keep the compiler from loading every
                // coefficient of every polynomial at once, which spills registers)
                const float dMcf = df_round(df_dot<11>(Ef + EV_PM, b11));
                asm volatile("" ::: "memory");
                const float dEtf = df_round(df_dot<11>(Ef + EV_PE, b11));
                asm volatile("" ::: "memory");
                float d9 = 0.0f, d10 = 0.0f;
                if (NP == 11) {
                    const DF b4[4] = {vi2, vinv, v5, v7};
                    d9 = df_round(df_dot<4>(Ef + EV_P9, b4));
                    d10 = df_round(df_dot<4>(Ef + EV_P10, b4));
                    asm volatile("" ::: "memory");
                }
                DF tau = DF{0.0f, 0.0f};
                float tMc = 0.0f, tEt = 0.0f;
                if (ROT) {
                    const DF b8[8] = {vi5, vi3, vi2, vinv, one, v, v2, vl};
                    tau = df_mul(df_dot<8>(Ef + EV_T0, b8), vi3);
                    asm volatile("" ::: "memory");
                    tMc = (float)OMEGA_E * df_round(df_mul(df_dot<8>(Ef + EV_TM, b8), vi3));
                    asm volatile("" ::: "memory");
                    tEt = (float)OMEGA_E * df_round(df_mul(df_dot<8>(Ef + EV_TE, b8), vi3));
                    asm volatile("" ::: "memory");
                }
                const DF fdf = df_mul(v3, inv_pim);
                const float ff = df_round(fdf);
                const float twopif = (float)TWO_PI * ff;

                // ---------------- FP32: noise weight and amplitude per PSD
                const float w = ff * (k == 0 ? wc0 : (k == N - 1 ? wcn : wcm));
                float sig[MAX_PSD];
#pragma unroll
                for (int p = 0; p < MAX_PSD; p++) {
                    if (p < net.n_psd) {
                        const float x = ff * net.psd_inv_f0_f[p];
                        const float xi = 1.0f / x;
                        float S = 0.0f;
                        for (int q = 0; q < net.psd_nterm[p]; q++) {
                            const int pw = net.psd_pow[p][q];
                            S = fmaf(net.psd_coef_f[p][q], pw >= 0 ? ipowf(x, pw) : ipowf(xi, -pw), S);
                        }
                        sig[p] = Aamp * sqrtf(4.0f * w / S);
                    } else {
                        sig[p] = 0.0f;
                    }
                }

#pragma unroll 1
                for (int s = 0; s < net.n_site; s++) {
                    const float *S = A.sitec_f + (e * net.n_site + s) * (int64_t)SC_N;
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
                    for (int q = net.site_ifo0[s]; q < net.site_ifo1[s]; q++) {
                        const float amp = (float)net.ifo_amp[q];
                        const PatF pt = patterns_f((float)net.ifo_s2g[q], (float)net.ifo_c2g[q],
                                                   amp * c2p, amp * s2p, J);
                        const float sg = sig[net.ifo_psd[q]];
                        float gr[NP], gi[NP], qr, qi, xr, xi, tr, ti;
                        tangents_f<NP, ROT>(pt, sg * cp, sg * cx, sg * dcp, sg * dcx, aMc, invdL,
                                            ph, gr, gi, qr, qi, xr, xi, tr, ti);
                        // tangents as (real, imaginary) pairs and their negations
                        float2 G[NP], NG[NP];
#pragma unroll
                        for (int i = 0; i < NP; i++) {
                            G[i] = make_float2(gr[i], gi[i]);
                            NG[i] = make_float2(-gr[i], -gi[i]);
                        }
                        const float2 Q = make_float2(qr, qi);
                        if (MODE == MODE_FISHER) {
                            // Gamma_ij: real and imaginary products summed separately
                            // (|Q|^2 = the (Phic, Phic) entry, copied at the end)
                            int a = 1;
#pragma unroll
                            for (int i = 0; i < NP; i++) {
#pragma unroll
                                for (int jj = i; jj < NP; jj++) {
                                    acc_pk(acc[a], mylo + a * NT, G[i], G[jj], NG[jj]);
                                    a++;
                                }
                                if (i & 1) asm volatile("" ::: "memory");
                            }
                            // phase-free SNR-gradient sums (see N_SNRGRAD_X)
                            constexpr int X0 = 1 + NP * (NP + 1) / 2;
                            const float2 X = make_float2(xr, xi), NX = make_float2(-xr, -xi);
                            const float2 T = make_float2(tr, ti), NT2 = make_float2(-tr, -ti);
                            acc_pk(acc[X0 + 0], mylo + (X0 + 0) * NT, Q, X, NX);
                            acc_pk(acc[X0 + 1], mylo + (X0 + 1) * NT,
                                   make_float2(ph.tMc * qr, ph.tMc * qi), X, NX);
                            acc_pk(acc[X0 + 2], mylo + (X0 + 2) * NT,
                                   make_float2(ph.teta * qr, ph.teta * qi), X, NX);
                            acc_pk(acc[X0 + 3], mylo + (X0 + 3) * NT, Q, T, NT2);
                            acc_pk(acc[X0 + 4], mylo + (X0 + 4) * NT, Q, G[5], NG[5]);
                            acc_pk(acc[X0 + 5], mylo + (X0 + 5) * NT, Q, G[6], NG[6]);
                        } else if (MODE == MODE_SNR) {
                            const float2 NQ = make_float2(-qr, -qi);
                            acc_pk(acc[0], mylo, Q, Q, NQ);
                            const int dd = net.ifo_det[q];
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd) acc_pk(acc[1 + d], mylo + (1 + d) * NT, Q, Q, NQ);
                        } else {   // MODE_SNRGRAD
                            const float2 NQ = make_float2(-qr, -qi);
                            acc_pk(acc[0], mylo, Q, Q, NQ);
#pragma unroll
                            for (int i = 0; i < 8; i++)
                                acc_pk(acc[1 + i], mylo + (1 + i) * NT, Q, G[i], NG[i]);
                        }
                    }
                }
                v = df_mul(v, rho);
                vinv = df_mul(vinv, rhoi);
                lnv = df_add(lnv, dlnv);
                Aamp *= rA;
            }
        }
        // ---- group reduction: butterfly over the GROUP lanes in double-float
        // (error-free two-sum of the high parts, compensations added), then
        // every lane writes the accumulators a = gl (mod GROUP) in FP64
        double *out = A.partial + it * (int64_t)A.nacc;
        if (MODE == MODE_FISHER) {
            // SNR^2 = sum |Q|^2 = the (Phic, Phic) entry
            constexpr int k88 = 1 + 8 * NP - 8 * 7 / 2;
            acc[0] = acc[k88];
            mylo[0] = mylo[k88 * NT];
        }
#pragma unroll
        for (int a = 0; a < NACC; a++) {
            // collapse (real, imaginary) parts: value = -(hn.x + hn.y + ln.x + ln.y)
            const float2 l2 = mylo[a * NT];
            const DF h = two_sum(acc[a].x, acc[a].y);
            DF s = DF{-h.hi, -((l2.x + l2.y) + h.lo)};
#pragma unroll
            for (int o = 1; o < GROUP; o <<= 1) {
                const float oh = __shfl_xor_sync(gmask, s.hi, o);
                const float ol = __shfl_xor_sync(gmask, s.lo, o);
                // identical operands on both lanes of a pair: same result on both
                const DF t = (gl & o) ? two_sum(oh, s.hi) : two_sum(s.hi, oh);
                s.hi = t.hi;
                s.lo = ((gl & o) ? (ol + s.lo) : (s.lo + ol)) + t.lo;
            }
            if ((a % GROUP) == gl && a < A.nacc) out[a] = (double)s.hi + (double)s.lo;
        }
        __syncwarp(gmask);
    }
}

template <int MODE, int NP, bool ROT>
cudaError_t launch_one_m(const PointArgs &a, cudaStream_t s)
{
    constexpr int NACC = NAccM<MODE, NP>::value;
    const size_t smem = ((size_t)NACC * 128 + (size_t)4 * GROUPS_PER_WARP * EVC) * sizeof(float2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t err = cudaFuncSetAttribute(k_points_mixed<MODE, NP, ROT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        attr_set = true;
    }
    if (a.n_items <= 0) return cudaSuccess;
    k_points_mixed<MODE, NP, ROT><<<points_grid_size(2), 128, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode_m(int np, int rot, const PointArgs &a, cudaStream_t s)
{
    if (np == 9) return rot ? launch_one_m<MODE, 9, true>(a, s) : launch_one_m<MODE, 9, false>(a, s);
    return rot ? launch_one_m<MODE, 11, true>(a, s) : launch_one_m<MODE, 11, false>(a, s);
}

}  // namespace

cudaError_t launch_points_mixed(int mode, int np, int rot, const PointArgs &a, cudaStream_t s)
{
    switch (mode) {
    case MODE_SNR: return launch_mode_m<MODE_SNR>(np, rot, a, s);
    case MODE_FISHER: return launch_mode_m<MODE_FISHER>(np, rot, a, s);
    default: return launch_mode_m<MODE_SNRGRAD>(np, rot, a, s);
    }
}

}  // namespace gw
