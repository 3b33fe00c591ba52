// gw_kernels.cuh -- launch interfaces between the host API (gw_api.cu) and the
// kernels (gw_setup.cu, gw_points_fp64.cu, gw_points_mixed.cu).
#pragma once

#include <atomic>

#include "gw_internal.cuh"

namespace gw {

// ---- per-device launch facts.  cudaFuncSetAttribute acts on the current
// device only, and the SM count sizes the persistent grids, so both are kept
// per device (devices 0..63; beyond that they are taken on every launch).
constexpr int MAX_CACHED_DEV = 64;

inline int current_device()
{
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess ? dev : 0;
}

// the network has a tabulated PSD (the point kernels' table instantiation)
inline bool has_psd_table(const DevNet &net)
{
    for (int p = 0; p < net.n_psd; p++)
        if (net.psd_kind[p] == 1) return true;
    return false;
}

// one bit per device: the kernel's attribute has been set there
struct PerDeviceOnce {
    std::atomic<unsigned long long> bits{0};
};

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device and kernel
template <typename K>
cudaError_t set_smem_once(PerDeviceOnce &once, K kernel, size_t smem)
{
    const int dev = current_device();
    const unsigned long long bit = dev < MAX_CACHED_DEV ? 1ull << dev : 0ull;
    if (bit && (once.bits.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && bit) once.bits.fetch_or(bit, std::memory_order_release);
    return e;
}

// catalog in device memory (pointers may be null where the ABI allows)
struct DevCat {
    int64_t n;
    const double *Mc, *eta, *dL, *theta, *phi, *iota, *psi, *tc, *Phic;
    const double *chi1, *chi2, *LamT, *dLamT;
    const int8_t *pset;
    const double *fmin, *fmax;
    const int32_t *npts;
    const uint32_t *arm_mask;   // duty-factor arm masks per row, or null (all on)
    const int64_t *sel;         // rows of the call's events, or null (identity)
};

struct PointArgs {
    DevNet net;
    const double *evc;        // [n][EVC]
    const double *sitec;      // [n][n_site][SC_N]
    const float *sitec_f;     // [n][n_site][SC_N], FP32 copy for the mixed path
    const float2 *evc_f;      // [n][EVC], double-float copy for the mixed path
    const int64_t *item_off;  // [n+1] exclusive prefix of work items per event
    int64_t n_ev;
    int64_t n_items;          // capacity of partial in items; the kernels process
                              // min(item_off[n_ev], n_items) items
    double *partial;          // [n_items][nacc]
    int nacc;
    const double *cov;        // logdet mode: covariance, packed, event-minor
    uint32_t det_mask = 0xffffffffu;   // logdet mode: detectors whose orientation
                                       // gradient is formed (bit d); other sites skipped
    int group = GROUP;                 // Fisher pass: lanes per work item (4, 8 or 16)
    int blocks_per_sm = 2;             // persistent grid: CTAs per SM (1 or 2)
    int32_t *kerr = nullptr;           // set to 1 by a kernel whose bounded wait ran out
};

// extra accumulators of the mixed Fisher kernel: phase-free SNR-gradient sums
//   Re(Q* dQ/dx), Omega tau*_Mc Re(Q* dQ/dx), Omega tau*_eta Re(Q* dQ/dx),
//   Re(Q* dQ/dtheta), Re(Q* dQ/diota), Re(Q* dQ/dpsi)
constexpr int N_SNRGRAD_X = 6;

// number of accumulators per work item
inline int n_acc(int mode, int np, int n_det, bool mixed = false)
{
    switch (mode) {
    case MODE_SNR: return 1 + n_det;
    case MODE_FISHER: return 1 + np * (np + 1) / 2 + (mixed ? N_SNRGRAD_X : 0);
    case MODE_SNRGRAD: return 1 + np + n_det;
    default: return n_det;
    }
}

cudaError_t launch_prepare(int64_t n, const double *m1, const double *m2, const double *chi1,
                           const double *chi2, const double *lam1, const double *lam2,
                           const double *dL_Mpc, const uint8_t *zflag, const double *tcoal,
                           const double *fmin, const int32_t *npts_given, int32_t npts_fixed,
                           double per_efold, int32_t lo, int32_t hi, double *Mc, double *eta,
                           double *dL_Gpc, double *chi1o, double *chi2o, double *LamT,
                           double *dLamT, double *tc_s, double *fmax, int32_t *npts,
                           cudaStream_t s);

// event constants, status, and work items per event (items of at most
// `chunk` grid points: CHUNK_MAX, or TC_CHUNK for the tensor-core Fisher pass)
cudaError_t launch_event_setup(const DevCat &cat, const DevNet &net, int np, double *evc,
                               double *sitec, float *sitec_f, float2 *evc_f, int32_t *status,
                               int64_t *counts, cudaStream_t s, int chunk = CHUNK_MAX);

// exclusive scan of counts[0..n) into off[0..n], off[n] = total; tmp needs
// scan_tmp_size(n) int64 elements
size_t scan_tmp_size(int64_t n);
cudaError_t launch_scan(const int64_t *counts, int64_t n, int64_t *off, int64_t *tmp,
                        cudaStream_t s);

cudaError_t launch_points_fp64(int mode, int np, int rot, const PointArgs &a, cudaStream_t s);
// FP64 Fisher pass with the Gram on the tensor cores (gw_points_fp64_tc.cu):
// networks of at most two interferometers per grid point
bool fisher_fp64_tc_supported(const DevNet &net);
constexpr int TC_CHUNK = 128;   // points per work item of the tensor-core Fisher pass
cudaError_t launch_fisher_fp64_tc(int np, int rot, const PointArgs &a, cudaStream_t s);
// the same pass with the tangents in double-float on the FP32 pipe
cudaError_t launch_fisher_dfloat_tc(int np, int rot, const PointArgs &a, cudaStream_t s);
cudaError_t launch_points_mixed(int mode, int np, int rot, const PointArgs &a, cudaStream_t s);

// partial sums of the items of each event -> outputs
cudaError_t launch_finish(int mode, int np, int n_det, const PointArgs &a, const int32_t *status,
                          double *snr, double *snr_det, double *fisher, const double *grad_snr,
                          double *grad_params, double *grad_gamma, double *xsums, cudaStream_t s);

// SNR vector-Jacobian product from a Fisher pass (see gw_fisher)
// strain output (gw_strain.cu): off = exclusive scan of the events' grid lengths
cudaError_t launch_point_offsets(const int32_t *npts, const int64_t *sel, int64_t n,
                                 int64_t *counts, int64_t *off, int64_t *scan_tmp, cudaStream_t s);
cudaError_t launch_strain(const DevNet &net, int64_t n, int64_t total, int mixed,
                          const double *evc, const double *sitec, const int32_t *status,
                          const int64_t *poff, double *re, double *im, double *freq,
                          cudaStream_t s);

// covariance tools (gw_covtools.cu)
struct CovArgs {
    int64_t n;
    int P, Pk;             // parameters of the input, parameters kept
    int idx[11];           // kept parameter slots, increasing
    double prior[11];      // added to the diagonal, per original slot
    int method;            // gw_inv_method
    double thresh, cond_max;
};
struct SubIdx {
    int idx[11];
};
cudaError_t launch_fisher_eig(int64_t n, int P, int normalize, const double *F, double *w,
                              double *V, cudaStream_t s);
cudaError_t launch_covariance(const CovArgs &a, const double *F, double *cov, double *cond,
                              double *eps, int32_t *status, cudaStream_t s);
cudaError_t launch_submatrix(int64_t n, int P, int K, const SubIdx &idx, const double *in,
                             double *out, cudaStream_t s);
cudaError_t launch_perturb(int64_t total, double eps, const double *F, const double *r,
                           double *out, cudaStream_t s);
cudaError_t launch_sky_area(int64_t n, int P, int it, int ip, const double *cov,
                            const double *theta, double perc, int units, double *area,
                            cudaStream_t s);

// detection gate: sel = indices i with snr[i] > th (increasing); off[n] = count
cudaError_t launch_select(const double *snr, int64_t n, double th, int64_t *flag, int64_t *off,
                          int64_t *scan_tmp, int64_t *sel, cudaStream_t s);
cudaError_t launch_snr_grad_from_fisher(int64_t n, int np, bool mixed, int rot,
                                        const double *fisher, const double *snr,
                                        const double *xsums, const double *evc,
                                        const int32_t *status, const double *grad_snr,
                                        double *grad_params, cudaStream_t s);

// log table of a tabulated PSD (gw_setup.cu): nseg segments of (f, S) pairs
cudaError_t launch_psd_table(const double *f, const double *S, int64_t nseg, int is_asd,
                             double ln_scale, double ln_ref, PsdSeg *seg, float4 *segf,
                             cudaStream_t s);

// precision refinement (gw_refine.cu)
cudaError_t launch_refine_select(int64_t n, double cond_th, const int32_t *status,
                                 const int32_t *inv_status, const double *cond, const int64_t *sel,
                                 int64_t *flag, int64_t *off, int64_t *scan_tmp, int64_t *pos,
                                 int64_t *rows, uint8_t *refined, cudaStream_t s);
// the call's events split by parameter set (bit pset of mask: part a, else b):
// order-preserving positions and catalog rows of each part; flag, pos, rows
// [2n], off [2(n + 1)] (part b at offset n, its count at off[2n + 1])
cudaError_t launch_split_pset(int64_t n, const int8_t *pset, const int64_t *sel, uint32_t mask,
                              int64_t *flag, int64_t *off, int64_t *scan_tmp, int64_t *pos,
                              int64_t *rows, cudaStream_t s);
// part b's events to recompute with part a (k_flag_refine's rule on part b's
// m results, pos_b their call indices) marked in part a's flags, then part a
// compacted again: off_a [n + 1] (its new count at off_a[n]), pos_a, rows_a [n]
cudaError_t launch_route_recompute(int64_t m, double cond_th, const int32_t *status,
                                   const int32_t *inv_status, const double *cond,
                                   const int64_t *pos_b, int64_t n, const int64_t *sel,
                                   int64_t *flag_a, int64_t *off_a, int64_t *scan_tmp,
                                   int64_t *pos_a, int64_t *rows_a, cudaStream_t s);
cudaError_t launch_gather(int64_t m, const int64_t *pos, const double *in, double *out,
                          cudaStream_t s);
// event-minor arrays written back at positions pos of an n-event call: for
// each array of the set, out[k * n + pos[j]] = in[k * m + j], k < its rows,
// j < m; one launch for the whole set (elements of 8 or 4 bytes; an array
// with a null destination is left out)
struct ScatterSet {
    static constexpr int MAX = 8;
    int na = 0;
    int row0[MAX + 1] = {0};      // first row of each array in the set's rows
    int esz[MAX] = {0};
    const void *in[MAX] = {nullptr};
    void *out[MAX] = {nullptr};
    void add(const void *src, void *dst, int rows, int elem_bytes);
};
cudaError_t launch_scatter_set(int64_t m, int64_t n, const int64_t *pos, const ScatterSet &set,
                               cudaStream_t s);

// out[r] = sum over e of x[r * n + e], r < rows (one block per row, fixed order)
cudaError_t launch_sum_events(const double *x, int64_t n, int rows, double *out, cudaStream_t s);

cudaError_t launch_invert(const double *fisher, int64_t n, int np, double cond_max, double *cov,
                          double *cond, double *inv_err, int32_t *status, cudaStream_t s);

int device_sm_count();                      // SM count of the current device (cached per device)
int points_grid_size(int blocks_per_sm);   // persistent grid (blocks) for the point kernels

}  // namespace gw
