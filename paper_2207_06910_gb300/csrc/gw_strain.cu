// gw_strain.cu -- the detector strain itself, h_a(f_k) = Q_a(f_k) exp(i Phi_a(f_k)),
// on every event's grid and every arm of the network (the signal of Sec. 2.2
// projected as in Sec. 3.1, with the Earth-rotation Doppler phase).
//
// The Fisher path never needs exp(i Phi) (the phase cancels in Re(d_i h^* d_j h)),
// so this is an output tool.  The phase Phi = Psi(f) - Phic - pi/4 + Phi_D(f)
// reaches 1e6 rad on the 2 Hz grids: it is evaluated in FP64 and reduced to
// [-pi, pi] by the Cody-Waite method (W. J. Cody and W. Waite, Software Manual
// for the Elementary Functions, 1980): 2 pi is split into C1 + C2 + C3 with C1
// holding 24 significant bits, so that k C1 is exact for |k| < 2^29 and the
// reduction loses nothing to cancellation.  The reduced angle goes through
// FP64 sincos (GW_FP64) or FP32 sincosf (GW_MIXED).
#include <cmath>

#include "gw_kernels.cuh"

namespace gw {

namespace {

// 2 pi = C1 + C2 + C3: C1 is 2 pi rounded to 24 significant bits, C2 the
// remainder rounded to double, C3 the remainder of that
constexpr double TWO_PI_C1 = 0x1.921fb6p+2;
constexpr double TWO_PI_C2 = -0x1.777a5cf72cecep-23;
constexpr double TWO_PI_C3 = -0x1.9d747f23e32edp-77;

__device__ __forceinline__ double reduce_2pi(double x)
{
    const double k = rint(x * (1.0 / TWO_PI));
    double r = fma(-k, TWO_PI_C1, x);     // exact: k C1 has <= 53 bits and r is small
    r = fma(-k, TWO_PI_C2, r);
    return fma(-k, TWO_PI_C3, r);
}

__device__ __forceinline__ int64_t find_event_s(const int64_t *off, int64_t n, int64_t p)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_strain(DevNet net, int64_t n, int64_t total, int mixed, const double *evc,
                         const double *sitec, const int32_t *status, const int64_t *poff,
                         double *re, double *im, double *freq)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = find_event_s(poff, n, p);
        const int k = (int)(p - poff[e]);
        if (status[e] != 0) {
            for (int a = 0; a < net.n_arm; a++) re[a * total + p] = im[a * total + p] = NAN;
            if (freq) freq[p] = NAN;
            continue;
        }
        const double *E = evc + e * (int64_t)EVC;
        const double lnf = fma((double)k, E[EV_LNR], E[EV_LNF0]);
        const double f = exp(lnf);
        const double lnv = (lnf + E[EV_LNPIM]) * (1.0 / 3.0);
        const double v = exp(lnv), vi = exp(-lnv);
        const double vi2 = vi * vi, vi3 = vi2 * vi, vi5 = vi3 * vi2;
        const double v2 = v * v, v5 = v2 * v2 * v, v7 = v5 * v2;
        const double b11[11] = {vi5, vi3, vi2, vi, 1.0, v, v2, v5, v7, lnv, v * lnv};
        double psi = 0.0;
        for (int q = 10; q >= 0; q--) psi = fma(E[EV_PSI + q], b11[q], psi);
        double tau = 0.0;
        if (net.rotation) {
            const double b8[8] = {vi5, vi3, vi2, vi, 1.0, v, v2, v * lnv};
            for (int q = 7; q >= 0; q--) tau = fma(E[EV_T0 + q], b8[q], tau);
            tau *= vi3;
        }
        const double A = E[EV_A0] * exp(-7.0 / 6.0 * lnf);
        const double cp = E[EV_CP], cx = E[EV_CX], c2p = E[EV_C2PSI], s2p = E[EV_S2PSI];
        const uint32_t arm_on = (uint32_t)E[EV_ARMON];
        const double twopif = TWO_PI * f;
        if (freq) freq[p] = f;
        for (int s = 0; s < net.n_site; s++) {
            const double *S = sitec + (e * net.n_site + s) * (int64_t)SC_N;
            const double x = net.rotation ? fma(OMEGA_E, tau, S[SC_X0]) : S[SC_X0];
            double sx, cxx;
            sincos(x, &sx, &cxx);
            const double c2x = fma(2.0 * cxx, cxx, -1.0), s2x = 2.0 * sx * cxx;
            const double Ja = fma(S[SC_A1], c2x, fma(S[SC_A2], cxx, S[SC_A3]));
            const double Jb = fma(S[SC_A4], s2x, S[SC_A5] * sx);
            const double Jc = fma(S[SC_B1], c2x, S[SC_B2] * cxx);
            const double Jd = fma(S[SC_B3], s2x, S[SC_B4] * sx);
            const double phase = reduce_2pi(psi + E[EV_PHI0] +
                                            twopif * fma(S[SC_D1], cxx, S[SC_D2]));
            double sn, cs;
            if (mixed) {
                float sf, cf;
                sincosf((float)phase, &sf, &cf);
                sn = sf;
                cs = cf;
            } else {
                sincos(phase, &sn, &cs);
            }
            for (int q = net.site_ifo0[s]; q < net.site_ifo1[s]; q++) {
                const uint32_t need = net.ifo_need[q];
                if (need & (need - 1u)) continue;          // two-interferometer form: not an arm
                const int a = __ffs(need) - 1;
                const int64_t o = a * total + p;
                if (!((arm_on >> a) & 1u)) {                // arm off (duty factor): no data
                    re[o] = im[o] = 0.0;
                    continue;
                }
                const double s2g = net.ifo_s2g[q], c2g = net.ifo_c2g[q];
                const double aa = s2g * Ja + c2g * Jb, bb = c2g * Jc + s2g * Jd;
                const double amp = net.ifo_amp[q];
                const double fp = amp * (c2p * aa + s2p * bb), fx = amp * (c2p * bb - s2p * aa);
                const double qr = A * fp * cp, qi = A * fx * cx;
                re[o] = qr * cs - qi * sn;
                im[o] = qr * sn + qi * cs;
            }
        }
    }
}

__global__ void k_npts_counts(const int32_t *npts, const int64_t *sel, int64_t n, int64_t *counts)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) {
        const int N = npts[sel ? sel[e] : e];
        counts[e] = N > 0 ? N : 0;
    }
}

}  // namespace

cudaError_t launch_point_offsets(const int32_t *npts, const int64_t *sel, int64_t n,
                                 int64_t *counts, int64_t *off, int64_t *scan_tmp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_npts_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(npts, sel, n, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_scan(counts, n, off, scan_tmp, s);
}

cudaError_t launch_strain(const DevNet &net, int64_t n, int64_t total, int mixed,
                          const double *evc, const double *sitec, const int32_t *status,
                          const int64_t *poff, double *re, double *im, double *freq,
                          cudaStream_t s)
{
    if (n <= 0 || total <= 0) return cudaSuccess;
    const int bs = 256;
    int64_t nb = (total + bs - 1) / bs;
    if (nb > 152 * 64) nb = 152 * 64;
    k_strain<<<(unsigned)nb, bs, 0, s>>>(net, n, total, mixed, evc, sitec, status, poff, re, im,
                                         freq);
    return cudaGetLastError();
}

}  // namespace gw
