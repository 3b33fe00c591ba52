// gw_internal.cuh -- device-side data layout shared by the kernels of libgwfish.
//
// Per call, the host turns the caller's network into a DevNet passed by value
// as a kernel argument (it lives in the constant bank; every thread reads the
// same entries).  A triangle becomes two virtual 90-degree interferometers at
// bisectors gamma_T and gamma_T + 45 deg with amplitude 3/(2 sqrt 2): the three
// 60-degree arms (bisectors gamma_T + 30 + 120 k deg) have detector tensors
// that sum to zero, and the sum of the three arms' outer products of any
// quantity linear in the detector tensor (strain, its parameter derivatives)
// equals that of the two virtual interferometers.  This is exact, and replaces
// the paper's "third arm from the other two" saving (Sec. 3.3) by a two-term
// form: 2 of 3 projections and 2 of 3 rank-2 updates per point.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gw {

constexpr int MAX_SITE = 8;
constexpr int MAX_IFO = 24;
constexpr int MAX_ARM = 32;
constexpr int MAX_DET = 8;
constexpr int MAX_PSD = 4;
constexpr int MAX_TERM = 4;

// physical constants (SI; masses as G M / c^3 in seconds)
constexpr double PI = 3.141592653589793238462643383279502884;
constexpr double TWO_PI = 6.283185307179586476925286766559005768;
constexpr double EULER_GAMMA = 0.577215664901532860606512090082402431;
constexpr double T_SUN = 4.925490947641267e-6;
constexpr double C_SI = 299792458.0;
constexpr double MPC_M = 3.085677581491367e22;
constexpr double GPC_S = 1.0e3 * MPC_M / C_SI;
constexpr double R_EARTH_S = 6.371e6 / C_SI;       // Earth radius in light-seconds
constexpr double T_SIDEREAL = 86164.0905;
constexpr double OMEGA_E = TWO_PI / T_SIDEREAL;
constexpr double H0_KMS_MPC = 70.0;
constexpr double C_KMS = 299792.458;

// one segment of a tabulated PSD's log table (FP64 path)
struct __align__(32) PsdSeg {
    double lnf, lns, slope, lnf1;   // ln f_j, ln S_j, d ln S / d ln f, ln f_j+1
};

struct DevNet {
    int n_site, n_ifo, n_psd, rotation, n_det;
    int pad_;
    double site_slat[MAX_SITE], site_clat[MAX_SITE], site_lon[MAX_SITE];
    int site_ifo0[MAX_SITE], site_ifo1[MAX_SITE];   // IFOs of site s: [ifo0, ifo1)
    int ifo_site[MAX_IFO], ifo_psd[MAX_IFO], ifo_det[MAX_IFO];
    double ifo_s2g[MAX_IFO], ifo_c2g[MAX_IFO], ifo_amp[MAX_IFO];
    // duty factor: interferometer q is used for an event whose arm mask m has
    // (m & need) == need and not (excl != 0 and (m & excl) == excl).  A
    // triangle appears as its two-interferometer form (need = its three arms)
    // and as its three single arms (need = that arm, excl = its three arms).
    uint32_t ifo_need[MAX_IFO], ifo_excl[MAX_IFO];
    int site_nslot[MAX_SITE];   // interferometers in use per event and site: 1 (L), 2 (triangle)
    int n_arm;
    int masked;                 // the call has arm masks: read the slots per event
    double psd_inv_f0[MAX_PSD], psd_f0[MAX_PSD];
    int psd_nterm[MAX_PSD];
    double psd_coef[MAX_PSD][MAX_TERM];   // scale * coef
    int psd_pow[MAX_PSD][MAX_TERM];       // integer powers, |p| <= 15
    // FP32 path: PSDs divided by a reference scale (S_n ~ 1e-49 is below the
    // FP32 range) and the amplitude divided by sqrt(reference scale)
    float psd_coef_f[MAX_PSD][MAX_TERM];
    float psd_inv_f0_f[MAX_PSD];
    double inv_sqrt_scale_ref;
    double ln_scale_ref;                  // ln of the reference scale above
    // tabulated PSDs: segments psd_seg0[p] .. psd_seg0[p] + psd_nseg[p] - 1 of
    // psd_seg (FP64: ln f_j, ln S_j, slope, ln f_j+1, with S = scale x table)
    // and psd_seg_f (mixed path: two float4 per segment, ln f_j and
    // ln S_j - ln_scale_ref as double-float pairs, then slope, ln f_j+1 as a pair)
    int psd_kind[MAX_PSD];
    int psd_seg0[MAX_PSD], psd_nseg[MAX_PSD];
    const PsdSeg *psd_seg;
    const float4 *psd_seg_f;
};

// ---- per-event constants (FP64), row of EVC doubles per event ----------
enum EvSlot : int {
    EV_MC = 0, EV_ETA, EV_DL, EV_NPTS, EV_LNR,
    EV_WC0, EV_WCM, EV_WCN,            // trapezoid weight / f at first, interior, last point
    EV_LNF0,                            // ln fmin
    EV_LNPIM,                           // ln(pi M_s)
    EV_INV_PIM,                         // 1/(pi M_s)  (f = v^3 / (pi M_s))
    EV_PIM,                             // pi M_s      (1/f = pi M_s v^-3)
    EV_RHOG, EV_RHOIG, EV_LNRHOG,       // v, 1/v, ln v advance per GROUP points
    EV_A0,                              // A = A0 f^(-7/6)
    EV_RAG,                             // A advance per GROUP points
    EV_CP, EV_CX, EV_DCP, EV_DCX,       // (1+cos^2 i)/2, cos i and their iota derivatives
    EV_C2PSI, EV_S2PSI,
    EV_AMC,                             // 5 / (6 Mc)
    EV_INVDL,
    EV_IFOON,                           // bits of the interferometers in use (duty factor)
    EV_ARMON,                           // the event's arm mask (duty factor)
    EV_PHI0,                            // -Phic - pi/4 (strain phase constant)
    EV_PSI,                             // 11: Psi_PN + Psi_tidal      (basis B11)
    EV_PM = EV_PSI + 11,                // 11: d Psi / d Mc            (basis B11)
    EV_PE = EV_PM + 11,                 // 11: d Psi / d eta | Mc      (basis B11)
    EV_P9 = EV_PE + 11,                 // 4: slot 9  (v^-2, v^-1, v^5, v^7)
    EV_P10 = EV_P9 + 4,                 // 4: slot 10
    EV_T0 = EV_P10 + 4,                 // 8: tau*                (basis B8, times v^-3)
    EV_TM = EV_T0 + 8,                  // 8: d tau*/d Mc
    EV_TE = EV_TM + 8,                  // 8: d tau*/d eta | Mc
    EV_COEF_END = EV_TE + 8,
    EV_ADV = EV_COEF_END,               // 8: (rho, 1/rho, ln rho, amplitude ratio) of
                                        // v over 4 points, then over 16 points
    EVC = EV_ADV + 8
};
constexpr int NCOEF = EV_COEF_END - EV_PM;   // polynomial coefficients of the point loop
constexpr int NSCAL = EV_INVDL - EV_WC0 + 1;   // scalar constants of the mixed point loop
// B11 = (v^-5, v^-3, v^-2, v^-1, 1, v, v^2, v^5, v^7, ln v, v ln v)
// B8  = (v^-5, v^-3, v^-2, v^-1, 1, v, v^2, v ln v)

// ---- per (event, site) constants -----------------------------------------
enum SiteSlot : int {
    SC_X0 = 0,                    // phi - lon - Omega_E tc, reduced to [-pi, pi]
    SC_A1, SC_A2, SC_A3, SC_A4, SC_A5, SC_B1, SC_B2, SC_B3, SC_B4,
    SC_A1T, SC_A2T, SC_A3T, SC_A4T, SC_A5T, SC_B1T, SC_B2T, SC_B3T, SC_B4T,
    SC_D1, SC_D2, SC_D1T, SC_D2T, // Doppler: R/c [cos lat sin th, sin lat cos th] and d/d theta
    SC_SLOT0, SC_SLOT1,           // the interferometer entries in use (duty factor), -1 = none
    SC_X0LO,                      // FP32 table only: x0 - (float)x0 (double-float x0)
    SC_N
};

// accumulator layouts
template <int NP> struct Acc {
    static constexpr int NPAIR = NP * (NP + 1) / 2;
};

enum Mode : int { MODE_SNR = 0, MODE_FISHER = 1, MODE_SNRGRAD = 2, MODE_LOGDET = 3 };

// A work item is a contiguous run of at most CHUNK_MAX grid points of one
// event, processed by a group of G lanes (lane l takes points k0 + l,
// k0 + l + G, ...); a warp runs 32 / G items at once.  G = 8 by default: short
// items (the 200-300-point grids of light catalogs) then give every lane ~30
// points, which amortises the per-lane start and the per-item reduction; the
// Fisher point kernels are also built for G = 4 and 16 (the autotuner's choice).
constexpr int GROUP = 8;
constexpr int GROUPS_PER_WARP = 32 / GROUP;
constexpr int CHUNK_MAX = 256;                // points per work item (max)

// slot of recurrence factor k (0: rho = v ratio, 1: 1/rho, 2: ln rho, 3: amplitude
// ratio) over G points
template <int G>
__host__ __device__ constexpr int adv_slot(int k)
{
    return G == 8 ? (k == 0 ? EV_RHOG : k == 1 ? EV_RHOIG : k == 2 ? EV_LNRHOG : EV_RAG)
                  : EV_ADV + (G == 4 ? 0 : 4) + k;
}

}  // namespace gw
