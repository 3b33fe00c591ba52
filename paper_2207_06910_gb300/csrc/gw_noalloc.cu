// gw_noalloc.cu -- gw_fisher_noalloc: the Fisher / SNR pass without any memory
// allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example an application that gives all device memory to its own
// fixed-size pool at start-up (a cudaMalloc would then fail, or take memory
// the pool counts on), or a long-running or latency-bound loop that cannot
// afford an allocation's latency, its implicit synchronisation or its
// possible failure halfway through a job.  gw_fisher allocates its workspace
// lazily inside a gw_ctx, so those callers cannot use it.
//
// How: the workspace (per-event constants, work-item offsets, per-item partial
// sums) is carved out of one file-scope __device__ array of GW_NOALLOC_SCRATCH
// bytes that every GPU loading the library holds until the process exits.
// Host code cannot use the array's symbol as an address; its device address
// is obtained once per device with cudaGetSymbolAddress (on the first call on
// that device, with that device current, so that first call belongs before
// any stream capture) and passed to the kernels.  The kernels are the ones
// gw_fisher runs; every scratch word they read in a call is written earlier in
// the same call, so the previous call's contents never matter.  All calls
// share the array: calls whose work overlaps on the GPU (concurrent streams,
// or several host threads) race on it and must be serialised by the caller.
#include <cstdio>
#include <mutex>

#include "../../include/gwfish.h"
#include "gw_kernels.cuh"

using namespace gw;

// helpers of gw_api.cu (network expansion, tabulated PSDs, catalog checks)
gw_status gwi_build_net(gw_ctx *ctx, const gw_network *net, DevNet &d);
int64_t gwi_psd_segments(const DevNet &d);
cudaError_t gwi_prep_psd(const gw_network *net, DevNet &d, PsdSeg *seg, float4 *segf,
                         cudaStream_t s);
gw_status gwi_check_cat(gw_ctx *ctx, const gw_catalog *c, int np);
DevCat gwi_dev_cat(const gw_catalog *c);

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)GW_NOALLOC_SCRATCH_MIB << 20;
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[MAX_DEVICES] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// bump allocator over the static array: only hands out sub-ranges of it
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <typename T>
    T *take(size_t count)
    {
        T *p = reinterpret_cast<T *>(base + used);
        used += align256(count * sizeof(T));
        return p;
    }
};

}  // namespace

extern "C" gw_status gw_fisher_noalloc(const gw_catalog *cat, const gw_network *net,
                                       gw_precision prec, int n_par, double *fisher,
                                       double *snr, int32_t *status, void *stream)
{
    if (n_par != 9 && n_par != 11) return GW_EINVAL;
    if (prec != GW_FP64 && prec != GW_MIXED) return GW_EINVAL;
    gw_status st = gwi_check_cat(nullptr, cat, n_par);
    if (st) return st;
    DevNet dn;
    if ((st = gwi_build_net(nullptr, net, dn))) return st;
    dn.masked = cat->arm_mask != nullptr;
    const int64_t n = cat->n;
    if (n == 0) return GW_OK;
    if (!fisher || !status) return GW_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GW_ECUDA;
    {
        // one-time set-up per device: the device address of the static array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return GW_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool mixed = prec == GW_MIXED;
    const int nacc = n_acc(MODE_FISHER, n_par, dn.n_det, mixed);

    Carve c{g_scratch_ptr[dev]};
    double *evc = c.take<double>((size_t)n * EVC);
    double *sitec = c.take<double>((size_t)n * dn.n_site * SC_N);
    float *sitec_f = mixed ? c.take<float>((size_t)n * dn.n_site * SC_N) : nullptr;
    float2 *evc_f = mixed ? c.take<float2>((size_t)n * EVC) : nullptr;
    int64_t *counts = c.take<int64_t>((size_t)n);
    int64_t *off = c.take<int64_t>((size_t)n + 1);
    int64_t *scan = c.take<int64_t>(scan_tmp_size(n));
    const int64_t nseg = gwi_psd_segments(dn);
    PsdSeg *pseg = nseg ? c.take<PsdSeg>((size_t)nseg) : nullptr;
    float4 *psegf = (nseg && mixed) ? c.take<float4>((size_t)2 * nseg) : nullptr;
    // the per-item partial sums take the rest; at least one item per event
    if (c.used + align256((size_t)n * nacc * sizeof(double)) > SCRATCH_BYTES) return GW_ETOOLARGE;

    if (nseg && gwi_prep_psd(net, dn, pseg, psegf, s) != cudaSuccess) return GW_ECUDA;
    const DevCat dc = gwi_dev_cat(cat);
    if (launch_event_setup(dc, dn, n_par, evc, sitec, sitec_f, evc_f, status, counts, s) !=
            cudaSuccess ||
        launch_scan(counts, n, off, scan, s) != cudaSuccess)
        return GW_ECUDA;
    int64_t n_items = 0;
    if (cudaMemcpyAsync(&n_items, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GW_ECUDA;
    const size_t need = c.used + align256((size_t)(n_items > 0 ? n_items : 1) * nacc * sizeof(double));
    if (need > SCRATCH_BYTES) return GW_ETOOLARGE;   // grids too long for the static workspace
    double *partial = c.take<double>((size_t)(n_items > 0 ? n_items : 1) * nacc);

    PointArgs pa;
    pa.net = dn;
    pa.evc = evc;
    pa.sitec = sitec;
    pa.sitec_f = sitec_f;
    pa.evc_f = evc_f;
    pa.item_off = off;
    pa.n_ev = n;
    pa.n_items = n_items;
    pa.partial = partial;
    pa.nacc = nacc;
    pa.cov = nullptr;
    cudaError_t e = mixed ? launch_points_mixed(MODE_FISHER, n_par, dn.rotation, pa, s)
                          : launch_points_fp64(MODE_FISHER, n_par, dn.rotation, pa, s);
    if (e != cudaSuccess) return GW_ECUDA;
    if (launch_finish(MODE_FISHER, n_par, dn.n_det, pa, status, snr, nullptr, fisher, nullptr,
                      nullptr, nullptr, nullptr, s) != cudaSuccess)
        return GW_ECUDA;
    return GW_OK;
}
