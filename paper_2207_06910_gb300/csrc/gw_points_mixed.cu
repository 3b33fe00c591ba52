// gw_points_mixed.cu -- the fused point loop in mixed precision.
//
// FP64: the log grid (v = (pi M f)^(1/3) and 1/v by recurrence, ln v), the
//       TaylorF2 phase derivatives d Psi/d theta_i, tau*(f) and its
//       derivatives, the Earth angle x = x0 + Omega_E tau* reduced to
//       [-pi, pi], and f itself.
// FP32: noise weight, amplitude, pattern functions, Doppler derivatives,
//       tangents g_i, and the products Re(g_i^* g_j).
// Sums: every product is split exactly (p = a b, e = fma(a, b, -p)) and added
//       to a double-float accumulator (hi, lo) with an error-free two-sum
//       (Knuth), so the accumulated Gamma_ij equals the exact sum of the FP32
//       products to ~1e-13 relative.  The only FP32 rounding left is that of the
//       tangents themselves, which perturbs Gamma like a slightly different
//       set of tangent vectors (a Gram matrix of perturbed vectors), not
//       element by element.
// The tangents are pre-scaled by sigma = A sqrt(4 w / S_n), so the weight is
// inside the products; a rounding of sigma is a common factor of all tangents
// of a point, i.e. a perturbation of the noise weight.
#include <cmath>

#include "gw_kernels.cuh"

namespace gw {

namespace {

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

// double-float accumulator: value = hi + lo
struct DF {
    float hi, lo;
};

// add a + b (two FP32 products given with their exact rounding errors ea, eb)
__device__ __forceinline__ void df_add2(DF &s, float a, float ea, float b, float eb)
{
    // p = a + b exactly as (p, ep)
    const float p = a + b;
    const float bb = p - a;
    const float ep = (a - (p - bb)) + (b - bb);
    // s.hi + p exactly as (t, et)
    const float t = s.hi + p;
    const float bq = t - s.hi;
    const float et = (s.hi - (t - bq)) + (p - bq);
    s.hi = t;
    s.lo += (ea + eb) + (ep + et);
}

template <int MODE, int NP>
struct NAccM {
    static constexpr int value = MODE == MODE_FISHER ? 1 + NP * (NP + 1) / 2
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
                                           float (&gr)[NP], float (&gi)[NP], float &qr, float &qi)
{
    const float omega = (float)OMEGA_E;
    qr = Acp * p.fp;
    qi = Acx * p.fx;
    const float xr = Acp * p.fpX, xi = Acx * p.fxX;
    const float tr = Acp * p.fpT, ti = Acx * p.fxT;
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
__global__ void __launch_bounds__(128) k_points_mixed(PointArgs A)
{
    constexpr int NACC = NAccM<MODE, NP>::value;
    extern __shared__ double red_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    double *red = red_smem + wib * (NACC * 33);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const DevNet &net = A.net;

    for (int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + wib; it < A.n_items;
         it += nwarps) {
        const int64_t e = find_event_m(A.item_off, A.n_ev, it);
        const int64_t j = it - A.item_off[e];
        const int64_t nj = A.item_off[e + 1] - A.item_off[e];
        const double *E = A.evc + e * (int64_t)EVC;
        const int N = (int)E[EV_NPTS];
        const int kb = (int)((int64_t)N * j / nj), ke = (int)((int64_t)N * (j + 1) / nj);

        DF acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; a++) acc[a] = DF{0.0f, 0.0f};

        int k = kb + lane;
        if (k < ke) {
            const double lnr = E[EV_LNR];
            const double lnf = fma((double)k, lnr, E[EV_LNF0]);
            double lnv = (lnf + E[EV_LNPIM]) * (1.0 / 3.0);
            double v = exp(lnv), vinv = exp(-lnv);
            float Aamp = (float)(E[EV_A0] * net.inv_sqrt_scale_ref * exp(-7.0 / 6.0 * lnf));
            const double rho = E[EV_RHO32], rhoi = E[EV_RHOI32], dlnv = E[EV_LNRHO32];
            const float rA = (float)E[EV_RA32];
            const double inv_pim = E[EV_INV_PIM];
            const float wc0 = (float)E[EV_WC0], wcm = (float)E[EV_WCM], wcn = (float)E[EV_WCN];
            const float cp = (float)E[EV_CP], cx = (float)E[EV_CX];
            const float dcp = (float)E[EV_DCP], dcx = (float)E[EV_DCX];
            const float c2p = (float)E[EV_C2PSI], s2p = (float)E[EV_S2PSI];
            const float aMc = (float)E[EV_AMC], invdL = (float)E[EV_INVDL];

            for (; k < ke; k += 32) {
                // ---------------- FP64 part
                const double vi2 = vinv * vinv, vi3 = vi2 * vinv, vi5 = vi3 * vi2;
                const double v2 = v * v, v5 = v2 * v2 * v, v7 = v5 * v2, vl = v * lnv;
                const double f = v2 * v * inv_pim;
                const double *PM = E + EV_PM, *PE = E + EV_PE;
                double dMc = PM[8] * v7;
                dMc = fma(PM[7], v5, dMc);
                dMc = fma(PM[10], vl, dMc);
                dMc = fma(PM[6], v2, dMc);
                dMc = fma(PM[5], v, dMc);
                dMc = PM[4] + dMc;
                dMc = fma(PM[3], vinv, dMc);
                dMc = fma(PM[2], vi2, dMc);
                dMc = fma(PM[1], vi3, dMc);
                dMc = fma(PM[0], vi5, dMc);
                double dEt = PE[8] * v7;
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
                float d9 = 0.0f, d10 = 0.0f;
                if (NP == 11) {
                    const double *P9 = E + EV_P9, *P10 = E + EV_P10;
                    d9 = (float)fma(P9[0], vi2, fma(P9[1], vinv, fma(P9[2], v5, P9[3] * v7)));
                    d10 = (float)fma(P10[0], vi2, fma(P10[1], vinv, fma(P10[2], v5, P10[3] * v7)));
                }
                double tau = 0.0;
                float tMc = 0.0f, tEt = 0.0f;
                if (ROT) {
                    const double *T0 = E + EV_T0, *TM = E + EV_TM, *TE = E + EV_TE;
                    const double b[8] = {vi5, vi3, vi2, vinv, 1.0, v, v2, vl};
                    double s0 = T0[7] * b[7], s1 = TM[7] * b[7], s2 = TE[7] * b[7];
#pragma unroll
                    for (int q = 6; q >= 0; q--) {
                        s0 = fma(T0[q], b[q], s0);
                        s1 = fma(TM[q], b[q], s1);
                        s2 = fma(TE[q], b[q], s2);
                    }
                    tau = s0 * vi3;
                    tMc = (float)(OMEGA_E * s1 * vi3);
                    tEt = (float)(OMEGA_E * s2 * vi3);
                }
                const float ff = (float)f;
                const float twopif = (float)(TWO_PI * f);
                const float dMcf = (float)dMc, dEtf = (float)dEt;

                // ---------------- FP32 part: weights and amplitude per PSD
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

                for (int s = 0; s < net.n_site; s++) {
                    const float *S = A.sitec_f + (e * net.n_site + s) * (int64_t)SC_N;
                    float xs;
                    if (ROT) {
                        double x = A.sitec[(e * net.n_site + s) * (int64_t)SC_N + SC_X0] +
                                   OMEGA_E * tau;
                        x -= TWO_PI * rint(x * (1.0 / TWO_PI));
                        xs = (float)x;
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
                        ph.Mc = ph.eta = ph.th = ph.ph = ph.tc = ph.p9 = ph.p10 = 0.0f;
                    }
                    for (int q = net.site_ifo0[s]; q < net.site_ifo1[s]; q++) {
                        const float amp = (float)net.ifo_amp[q];
                        const PatF pt = patterns_f((float)net.ifo_s2g[q], (float)net.ifo_c2g[q],
                                                   amp * c2p, amp * s2p, J);
                        const float sg = sig[net.ifo_psd[q]];
                        float gr[NP], gi[NP], qr, qi;
                        tangents_f<NP, ROT>(pt, sg * cp, sg * cx, sg * dcp, sg * dcx, aMc, invdL,
                                            ph, gr, gi, qr, qi);
                        {
                            const float p1 = qr * qr, p2 = qi * qi;
                            df_add2(acc[0], p1, fmaf(qr, qr, -p1), p2, fmaf(qi, qi, -p2));
                        }
                        if (MODE == MODE_FISHER) {
                            int a = 1;
#pragma unroll
                            for (int i = 0; i < NP; i++)
#pragma unroll
                                for (int jj = i; jj < NP; jj++) {
                                    const float p1 = gr[i] * gr[jj], p2 = gi[i] * gi[jj];
                                    df_add2(acc[a], p1, fmaf(gr[i], gr[jj], -p1), p2,
                                            fmaf(gi[i], gi[jj], -p2));
                                    a++;
                                }
                        } else if (MODE == MODE_SNR) {
                            const int dd = net.ifo_det[q];
                            const float p1 = qr * qr, p2 = qi * qi;
#pragma unroll
                            for (int d = 0; d < MAX_DET; d++)
                                if (d == dd)
                                    df_add2(acc[1 + d], p1, fmaf(qr, qr, -p1), p2,
                                            fmaf(qi, qi, -p2));
                        } else {   // MODE_SNRGRAD: phase parts left out (see FP64 kernel)
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                const float p1 = qr * gr[i], p2 = qi * gi[i];
                                df_add2(acc[1 + i], p1, fmaf(qr, gr[i], -p1), p2,
                                        fmaf(qi, gi[i], -p2));
                            }
                        }
                    }
                }
                v *= rho;
                vinv *= rhoi;
                lnv += dlnv;
                Aamp *= rA;
            }
        }
        // warp reduction in FP64 (hi + lo of every lane, fixed order); the PSD
        // reference scale cancels between sigma^2 and 1/S_n
#pragma unroll
        for (int a = 0; a < NACC; a++) red[a * 33 + lane] = (double)acc[a].hi + (double)acc[a].lo;
        __syncwarp();
        double *out = A.partial + it * (int64_t)A.nacc;
        for (int a = lane; a < A.nacc; a += 32) {
            double s = 0.0;
#pragma unroll 8
            for (int l = 0; l < 32; l++) s += red[a * 33 + l];
            out[a] = s;
        }
        __syncwarp();
    }
}

template <int MODE, int NP, bool ROT>
cudaError_t launch_one_m(const PointArgs &a, cudaStream_t s)
{
    constexpr int NACC = NAccM<MODE, NP>::value;
    const size_t smem = 4 * NACC * 33 * sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t err = cudaFuncSetAttribute(k_points_mixed<MODE, NP, ROT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        attr_set = true;
    }
    if (a.n_items <= 0) return cudaSuccess;
    k_points_mixed<MODE, NP, ROT><<<points_grid_size(), 128, smem, s>>>(a);
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
