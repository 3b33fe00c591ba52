// gw_refine.cu -- kernels of gw_fisher_refine and gw_fisher_routed: the
// events whose mixed-precision covariance is not determined to the mixed
// path's tolerance are selected by their condition number (Sec. 4.1: the
// conditioning check of the inversion), recomputed by the FP64 path
// (gw_fisher_refine) or the double-float path (gw_fisher_routed, which also
// splits a call's events by parameter set), and written back in place.
//
// Why a condition-number test: the mixed path's Fisher matrix carries an
// elementwise error of ~1e-7 of sqrt(Gamma_ii Gamma_jj) (FP32 patterns,
// amplitudes and tangents); Gamma^-1 amplifies an elementwise error by up to
// the condition number, so above ~1e7 the marginalised errors sqrt(diag C)
// can move by more than 1e-3.  The FP64 path's elementwise error is ~1e-14
// and keeps sqrt(diag C) within ~2e-16 kappa of the oracle.
#include "gw_kernels.cuh"

namespace gw {
namespace {

constexpr int BS = 256;

// flag[i] = event i (of the call) is refined: its point-loop status is clean
// and its mixed inversion failed, or its condition number exceeds cond_th;
// refined[i] (optional) records the decision
__global__ void k_flag_refine(int64_t n, double cond_th, const int32_t *status,
                              const int32_t *inv_status, const double *cond, int64_t *flag,
                              uint8_t *refined)
{
    const int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (i >= n) return;
    const bool inv_bad = (inv_status[i] & (1 | 4)) != 0;   // NOT_PD, NONFINITE
    const bool f = status[i] == 0 && (inv_bad || !(cond[i] <= cond_th));
    flag[i] = f ? 1 : 0;
    if (refined) refined[i] = f ? 1 : 0;
}

// order-preserving compaction: pos[j] = the call's index of the j-th flagged
// event, rows[j] = its catalog row (through the call's own selection)
__global__ void k_compact_flagged(int64_t n, const int64_t *flag, const int64_t *off,
                                  const int64_t *sel, int64_t *pos, int64_t *rows)
{
    const int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (i >= n || !flag[i]) return;
    const int64_t j = off[i];
    pos[j] = i;
    rows[j] = sel ? sel[i] : i;
}

// the recomputation rule of k_flag_refine on the m events of a part, marked
// in the other part's flags at the call's indices pos[j]: flag[pos[j]] = 1
// for each event to recompute (the other entries are left as they are)
__global__ void k_mark_refine(int64_t m, double cond_th, const int32_t *status,
                              const int32_t *inv_status, const double *cond, const int64_t *pos,
                              int64_t *flag)
{
    const int64_t j = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (j >= m) return;
    const bool inv_bad = (inv_status[j] & (1 | 4)) != 0;   // NOT_PD, NONFINITE
    if (status[j] == 0 && (inv_bad || !(cond[j] <= cond_th))) flag[pos[j]] = 1;
}

// the call's events by parameter set: flag_a[i] = 1 when bit pset of mask is
// set for event i's row, flag_b[i] the complement
__global__ void k_flag_pset(int64_t n, const int8_t *pset, const int64_t *sel, uint32_t mask,
                            int64_t *flag_a, int64_t *flag_b)
{
    const int64_t i = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (i >= n) return;
    const int p = pset ? (int)pset[sel ? sel[i] : i] : 0;
    const bool a = p >= 0 && p < 32 && ((mask >> p) & 1u);
    flag_a[i] = a ? 1 : 0;
    flag_b[i] = a ? 0 : 1;
}

__global__ void k_gather(int64_t m, const int64_t *pos, const double *in, double *out)
{
    const int64_t j = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (j < m) out[j] = in[pos[j]];
}

// out_a[k * n + pos[j]] = in_a[k * m + j] for every array a of the set and
// k < its rows (event-minor arrays): one thread per (row of the set, event),
// so that the loads of a warp are independent and coalesced
__global__ void k_scatter_set(int64_t m, int64_t n, const int64_t *__restrict__ pos,
                              ScatterSet set)
{
    const int64_t j = blockIdx.x * (int64_t)BS + threadIdx.x;
    if (j >= m) return;
    const int r = blockIdx.y;
    int a = 0;
    while (a + 1 < set.na && r >= set.row0[a + 1]) a++;
    const int64_t k = r - set.row0[a];
    const int64_t i = pos[j];
    if (set.esz[a] == 8)
        static_cast<double *>(set.out[a])[k * n + i] =
            static_cast<const double *>(set.in[a])[k * m + j];
    else
        static_cast<int32_t *>(set.out[a])[k * n + i] =
            static_cast<const int32_t *>(set.in[a])[k * m + j];
}

unsigned blocks(int64_t n) { return (unsigned)((n + BS - 1) / BS); }

}  // namespace

cudaError_t launch_refine_select(int64_t n, double cond_th, const int32_t *status,
                                 const int32_t *inv_status, const double *cond, const int64_t *sel,
                                 int64_t *flag, int64_t *off, int64_t *scan_tmp, int64_t *pos,
                                 int64_t *rows, uint8_t *refined, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_flag_refine<<<blocks(n), BS, 0, s>>>(n, cond_th, status, inv_status, cond, flag, refined);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_scan(flag, n, off, scan_tmp, s)) != cudaSuccess) return e;
    k_compact_flagged<<<blocks(n), BS, 0, s>>>(n, flag, off, sel, pos, rows);
    return cudaGetLastError();
}

cudaError_t launch_route_recompute(int64_t m, double cond_th, const int32_t *status,
                                   const int32_t *inv_status, const double *cond,
                                   const int64_t *pos_b, int64_t n, const int64_t *sel,
                                   int64_t *flag_a, int64_t *off_a, int64_t *scan_tmp,
                                   int64_t *pos_a, int64_t *rows_a, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e;
    if (m > 0) {
        k_mark_refine<<<blocks(m), BS, 0, s>>>(m, cond_th, status, inv_status, cond, pos_b,
                                               flag_a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_scan(flag_a, n, off_a, scan_tmp, s)) != cudaSuccess) return e;
    k_compact_flagged<<<blocks(n), BS, 0, s>>>(n, flag_a, off_a, sel, pos_a, rows_a);
    return cudaGetLastError();
}

cudaError_t launch_split_pset(int64_t n, const int8_t *pset, const int64_t *sel, uint32_t mask,
                              int64_t *flag, int64_t *off, int64_t *scan_tmp, int64_t *pos,
                              int64_t *rows, cudaStream_t s)
{
    // flag, pos, rows: [2n]; off: [2(n + 1)]; part a first, part b at offset n
    if (n <= 0) return cudaSuccess;
    k_flag_pset<<<blocks(n), BS, 0, s>>>(n, pset, sel, mask, flag, flag + n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int part = 0; part < 2; part++) {
        int64_t *fl = flag + part * n, *of = off + part * (n + 1);
        if ((e = launch_scan(fl, n, of, scan_tmp, s)) != cudaSuccess) return e;
        k_compact_flagged<<<blocks(n), BS, 0, s>>>(n, fl, of, sel, pos + part * n, rows + part * n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gather(int64_t m, const int64_t *pos, const double *in, double *out,
                          cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_gather<<<blocks(m), BS, 0, s>>>(m, pos, in, out);
    return cudaGetLastError();
}

void ScatterSet::add(const void *src, void *dst, int rows, int elem_bytes)
{
    if (!dst || rows <= 0 || na >= MAX) return;
    in[na] = src;
    out[na] = dst;
    esz[na] = elem_bytes;
    row0[na + 1] = row0[na] + rows;
    na++;
}

cudaError_t launch_scatter_set(int64_t m, int64_t n, const int64_t *pos, const ScatterSet &set,
                               cudaStream_t s)
{
    if (m <= 0 || set.na == 0) return cudaSuccess;
    const dim3 grid(blocks(m), (unsigned)set.row0[set.na]);
    k_scatter_set<<<grid, BS, 0, s>>>(m, n, pos, set);
    return cudaGetLastError();
}

}  // namespace gw
