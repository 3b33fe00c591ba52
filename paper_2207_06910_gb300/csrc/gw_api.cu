// gw_api.cu -- the C ABI of libgwfish (declared in include/gwfish.h):
// argument validation, network expansion, workspace management and the
// launch sequence  event setup -> work-item scan -> point loop -> reduction.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/gwfish.h"
#include "gw_kernels.cuh"

using namespace gw;

struct gw_ctx {
    int device = 0;
    char err[512] = {0};
    double *evc = nullptr;      size_t evc_cap = 0;
    double *sitec = nullptr;    size_t sitec_cap = 0;
    float *sitec_f = nullptr;   size_t sitec_f_cap = 0;
    float2 *evc_f = nullptr;    size_t evc_f_cap = 0;
    int32_t *status = nullptr;  size_t status_cap = 0;
    int64_t *counts = nullptr;  size_t counts_cap = 0;
    int64_t *off = nullptr;     size_t off_cap = 0;
    int64_t *scan = nullptr;    size_t scan_cap = 0;
    double *partial = nullptr;  size_t partial_cap = 0;
    double *xsums = nullptr;    size_t xsums_cap = 0;   // mixed SNR-gradient sums [6][n]
    double *snr_tmp = nullptr;  size_t snr_tmp_cap = 0;
    PsdSeg *psd_seg = nullptr;  size_t psd_seg_cap = 0;   // tabulated PSDs, FP64
    float4 *psd_seg_f = nullptr; size_t psd_seg_f_cap = 0;   // and the FP32 pairs
    // gw_fisher_refine: selection and the FP64 results of the refined events
    int64_t *ref_flag = nullptr;  size_t ref_flag_cap = 0;
    int64_t *ref_off = nullptr;   size_t ref_off_cap = 0;
    int64_t *ref_scan = nullptr;  size_t ref_scan_cap = 0;
    int64_t *ref_pos = nullptr;   size_t ref_pos_cap = 0;
    int64_t *ref_rows = nullptr;  size_t ref_rows_cap = 0;
    double *ref_F = nullptr;      size_t ref_F_cap = 0;
    double *ref_C = nullptr;      size_t ref_C_cap = 0;
    double *ref_g = nullptr;      size_t ref_g_cap = 0;
    double *ref_v = nullptr;      size_t ref_v_cap = 0;     // snr, grad_snr, cond, inv_err
    int32_t *ref_st = nullptr;    size_t ref_st_cap = 0;    // status, inverse status
    // gw_fisher_routed: the split by parameter set and both parts' results
    int64_t *rt_flag = nullptr;   size_t rt_flag_cap = 0;
    int64_t *rt_off = nullptr;    size_t rt_off_cap = 0;
    int64_t *rt_scan = nullptr;   size_t rt_scan_cap = 0;
    int64_t *rt_pos = nullptr;    size_t rt_pos_cap = 0;
    int64_t *rt_rows = nullptr;   size_t rt_rows_cap = 0;
    double *rt_F = nullptr;       size_t rt_F_cap = 0;
    double *rt_C = nullptr;       size_t rt_C_cap = 0;
    double *rt_g = nullptr;       size_t rt_g_cap = 0;
    double *rt_v = nullptr;       size_t rt_v_cap = 0;      // snr, grad_snr, cond, inv_err
    int32_t *rt_st = nullptr;     size_t rt_st_cap = 0;     // status, inverse status
    int64_t *h_total = nullptr;   // pinned
    int64_t item_cap = 0;       // > 0: asynchronous mode with this many work items
    int64_t reserved_events = 0;
    // Fisher-pass tile per precision and grid-length class (gw_set_tile,
    // gw_autotune): lanes per work item and CTAs per SM
    int tile_group[2][3] = {{GROUP, GROUP, GROUP}, {GROUP, GROUP, GROUP}};
    int tile_bps[2][3] = {{2, 2, 2}, {2, 2, 2}};
    int fp64_gram_tc = 0;       // FP64 Fisher pass: Gram on the tensor cores where supported
    int32_t *kerr = nullptr;    // device flag: a kernel's bounded wait ran out
    int profiling = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ev_recorded = false;
};

namespace {

// grid-length class of a call from its mean work items per event (items of
// GW_ITEM_POINTS points): 0 up to ~380 points, 1 up to ~3000, 2 beyond
int length_class(int64_t items, int64_t n)
{
    if (n <= 0) return 0;
    const double m = (double)items / (double)n;
    return m <= 1.5 ? 0 : (m <= 12.0 ? 1 : 2);
}

gw_status fail(gw_ctx *c, gw_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, GW_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                             \
    } while (0)

template <typename T>
gw_status ensure(gw_ctx *ctx, T *&p, size_t &cap, size_t need)
{
    if (need <= cap) return GW_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t n = need + need / 4 + 64;
    if (cudaMalloc((void **)&p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GW_ENOMEM, "workspace allocation of %zu bytes failed", n * sizeof(T));
    }
    cap = n;
    return GW_OK;
}

bool is_int(double x) { return std::isfinite(x) && std::fabs(x - std::nearbyint(x)) < 1e-12; }

}  // namespace

// network expansion and catalog checks, shared with the allocation-free entry
// point (gw_noalloc.cu); errors go to ctx when it is non-null
gw_status gwi_build_net(gw_ctx *ctx, const gw_network *net, DevNet &d)
{
    if (!net || !net->det || !net->psd) return fail(ctx, GW_EINVAL, "network: null pointer");
    if (net->n_det < 1 || net->n_det > MAX_DET)
        return fail(ctx, GW_EINVAL, "network: n_det=%d outside [1,%d]", net->n_det, MAX_DET);
    if (net->n_psd < 1 || net->n_psd > MAX_PSD)
        return fail(ctx, GW_EINVAL, "network: n_psd=%d outside [1,%d]", net->n_psd, MAX_PSD);
    memset(&d, 0, sizeof d);
    d.n_psd = net->n_psd;
    d.rotation = net->earth_rotation ? 1 : 0;
    d.n_det = net->n_det;
    // reference scale of the FP32 path: the first power-sum PSD's scale (S_n
    // ~ 1e-49 is below the FP32 range), else the first PSD's; tabulated PSDs
    // enter the FP32 path as ln S - ln(reference), never as S itself
    double scale_ref = 0.0;
    for (int p = 0; p < net->n_psd && scale_ref == 0.0; p++)
        if (net->psd[p].kind == GW_PSD_POWER_SUM) scale_ref = net->psd[p].scale;
    if (scale_ref == 0.0) scale_ref = net->psd[0].scale;
    int seg = 0;
    for (int p = 0; p < net->n_psd; p++) {
        const gw_psd &P = net->psd[p];
        if (!std::isfinite(P.scale) || P.scale <= 0)
            return fail(ctx, GW_EINVAL, "psd %d: need scale > 0", p);
        d.psd_kind[p] = P.kind;
        if (P.kind == GW_PSD_TABLE) {
            if (!P.table_f || !P.table_s || P.n_table < 2 || P.n_table > (1 << 20) ||
                (P.is_asd != 0 && P.is_asd != 1))
                return fail(ctx, GW_EINVAL, "psd %d: a table needs table_f, table_s, "
                            "2 <= n_table <= 2^20 and is_asd 0 or 1", p);
            d.psd_seg0[p] = seg;
            d.psd_nseg[p] = P.n_table - 1;
            seg += P.n_table - 1;
            continue;
        }
        if (P.kind != GW_PSD_POWER_SUM)
            return fail(ctx, GW_EINVAL, "psd %d: kind %d (0 = power sum, 1 = table)", p, P.kind);
        if (!(P.f0 > 0) || P.nterm < 1 || P.nterm > MAX_TERM)
            return fail(ctx, GW_EINVAL, "psd %d: need f0 > 0, 1 <= nterm <= 4", p);
        d.psd_f0[p] = P.f0;
        d.psd_inv_f0[p] = 1.0 / P.f0;
        d.psd_nterm[p] = P.nterm;
        for (int j = 0; j < P.nterm; j++) {
            if (!is_int(P.pw[j]) || std::fabs(P.pw[j]) > 15)
                return fail(ctx, GW_EUNSUPPORTED,
                            "psd %d term %d: power %g (only integer powers |p| <= 15)", p, j,
                            P.pw[j]);
            if (!std::isfinite(P.coef[j]) || P.coef[j] < 0)
                return fail(ctx, GW_EINVAL, "psd %d term %d: coefficient must be >= 0", p, j);
            d.psd_coef[p][j] = P.scale * P.coef[j];
            d.psd_coef_f[p][j] = (float)(P.scale / scale_ref * P.coef[j]);
            d.psd_pow[p][j] = (int)std::nearbyint(P.pw[j]);
        }
        d.psd_inv_f0_f[p] = (float)(1.0 / P.f0);
    }
    d.inv_sqrt_scale_ref = 1.0 / std::sqrt(scale_ref);
    d.ln_scale_ref = std::log(scale_ref);
    int ni = 0, na = 0;
    for (int s = 0; s < net->n_det; s++) {
        const gw_detector &D = net->det[s];
        if (!std::isfinite(D.lat) || !std::isfinite(D.lon) || !std::isfinite(D.gamma) ||
            !std::isfinite(D.zeta))
            return fail(ctx, GW_EINVAL, "detector %d: non-finite angle", s);
        if (D.shape != 0 && D.shape != 1)
            return fail(ctx, GW_EINVAL, "detector %d: shape %d (0 = L, 1 = triangle)", s, D.shape);
        if (D.psd < 0 || D.psd >= net->n_psd)
            return fail(ctx, GW_EINVAL, "detector %d: psd index %d", s, D.psd);
        d.site_slat[s] = std::sin(D.lat);
        d.site_clat[s] = std::cos(D.lat);
        d.site_lon[s] = D.lon;
        const int n_arms_s = D.shape == 0 ? 1 : 3;
        const int n_ifo_s = D.shape == 0 ? 1 : 5;
        if (na + n_arms_s > MAX_ARM || ni + n_ifo_s > MAX_IFO)
            return fail(ctx, GW_EUNSUPPORTED, "network: more than %d arms or %d interferometer "
                        "entries", MAX_ARM, MAX_IFO);
        d.site_ifo0[s] = ni;
        const uint32_t arms = ((1u << n_arms_s) - 1u) << na;
        auto add = [&](double g, double amp, uint32_t need, uint32_t excl) {
            d.ifo_s2g[ni] = std::sin(2.0 * g);
            d.ifo_c2g[ni] = std::cos(2.0 * g);
            d.ifo_amp[ni] = amp;
            d.ifo_site[ni] = s;
            d.ifo_psd[ni] = D.psd;
            d.ifo_det[ni] = s;
            d.ifo_need[ni] = need;
            d.ifo_excl[ni] = excl;
            ni++;
        };
        if (D.shape == 0) {
            add(D.gamma, std::sin(D.zeta), arms, 0u);
        } else {
            // every arm on: two virtual 90-degree interferometers at gamma_T and
            // gamma_T + 45 deg with amplitude sqrt(3/2) sin(60 deg) = 3/(2 sqrt 2)
            add(D.gamma, 1.5 / std::sqrt(2.0), arms, 0u);
            add(D.gamma + 0.25 * M_PI, 1.5 / std::sqrt(2.0), arms, 0u);
            // otherwise the arms that are on, each a 60-degree interferometer:
            // a 90-degree one at its bisector with amplitude sin(60 deg)
            for (int k = 0; k < 3; k++)
                add(D.gamma + M_PI / 6.0 + 2.0 * M_PI * k / 3.0, std::sqrt(3.0) / 2.0,
                    1u << (na + k), arms);
        }
        na += n_arms_s;
        d.site_ifo1[s] = ni;
        d.site_nslot[s] = D.shape == 0 ? 1 : 2;
    }
    d.n_site = net->n_det;
    d.n_ifo = ni;
    d.n_arm = na;
    return GW_OK;
}

// segments of the network's tabulated PSDs (0: none)
int64_t gwi_psd_segments(const DevNet &d)
{
    int64_t n = 0;
    for (int p = 0; p < d.n_psd; p++)
        if (d.psd_kind[p] == GW_PSD_TABLE) n += d.psd_nseg[p];
    return n;
}

// the device log tables of the network's tabulated PSDs, built into seg
// (FP64, gwi_psd_segments entries) and segf (two per segment; may be null
// when the mixed path is not used)
cudaError_t gwi_prep_psd(const gw_network *net, DevNet &d, PsdSeg *seg, float4 *segf,
                         cudaStream_t s)
{
    d.psd_seg = seg;
    d.psd_seg_f = segf;
    for (int p = 0; p < d.n_psd; p++) {
        if (d.psd_kind[p] != GW_PSD_TABLE) continue;
        const gw_psd &P = net->psd[p];
        cudaError_t e = launch_psd_table(P.table_f, P.table_s, d.psd_nseg[p], P.is_asd,
                                         std::log(P.scale), d.ln_scale_ref, seg + d.psd_seg0[p],
                                         segf ? segf + 2 * d.psd_seg0[p] : nullptr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

gw_status gwi_check_cat(gw_ctx *ctx, const gw_catalog *c, int np)
{
    if (!c) return fail(ctx, GW_EINVAL, "catalog: null");
    if (c->n < 0) return fail(ctx, GW_EINVAL, "catalog: n < 0");
    if (c->n == 0) return GW_OK;
    if (!c->Mc || !c->eta || !c->dL || !c->theta || !c->phi || !c->iota || !c->psi || !c->tc ||
        !c->Phic || !c->fmin || !c->fmax || !c->npts)
        return fail(ctx, GW_EINVAL, "catalog: a required array is null");
    if (np == 11 && !c->pset) return fail(ctx, GW_EINVAL, "catalog: n_par 11 needs pset");
    return GW_OK;
}

DevCat gwi_dev_cat(const gw_catalog *c)
{
    DevCat d;
    d.n = c->n;
    d.Mc = c->Mc; d.eta = c->eta; d.dL = c->dL; d.theta = c->theta; d.phi = c->phi;
    d.iota = c->iota; d.psi = c->psi; d.tc = c->tc; d.Phic = c->Phic;
    d.chi1 = c->chi1z; d.chi2 = c->chi2z; d.LamT = c->LamT; d.dLamT = c->dLamT;
    d.pset = c->pset; d.fmin = c->fmin; d.fmax = c->fmax; d.npts = c->npts;
    d.arm_mask = c->arm_mask; d.sel = c->sel;
    return d;
}

namespace {

// log-det gradient of an empty catalog: 0 for the selected detectors, NaN
// (all bits set) for the others
gw_status logdet_zero(gw_ctx *ctx, int n_det, uint32_t det_mask, double *grad_gamma,
                      cudaStream_t s)
{
    for (int d = 0; d < n_det; d++)
        CK(cudaMemsetAsync(grad_gamma + d, (det_mask >> d) & 1u ? 0 : 0xff, sizeof(double), s));
    return GW_OK;
}

// event setup -> scan -> point loop -> reduction
gw_status run_points(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                     int mode, int np, int32_t *status_out, double *snr, double *snr_det,
                     double *fisher, const double *grad_snr, double *grad_params,
                     const double *cov, double *grad_gamma, void *stream,
                     uint32_t det_mask = 0xffffffffu)
{
    cudaStream_t s = (cudaStream_t)stream;
    gw_status st = gwi_check_cat(ctx, cat, np);
    if (st) return st;
    if (np != 9 && np != 11) return fail(ctx, GW_EINVAL, "n_par must be 9 or 11 (got %d)", np);
    if (prec != GW_FP64 && prec != GW_MIXED && prec != GW_DFLOAT)
        return fail(ctx, GW_EINVAL, "bad precision");
    DevNet dn;
    if ((st = gwi_build_net(ctx, net, dn))) return st;
    dn.masked = cat->arm_mask != nullptr;
    const int64_t n = cat->n;
    const bool mixed = prec == GW_MIXED && (mode == MODE_FISHER || mode == MODE_SNR ||
                                            mode == MODE_SNRGRAD);
    const int nacc = n_acc(mode, np, dn.n_det, mixed);
    // fused SNR vector-Jacobian product of a Fisher pass
    const bool fused_grad = mode == MODE_FISHER && grad_params != nullptr;
    if (mode == MODE_LOGDET && !(det_mask & ((dn.n_det < 32 ? 1u << dn.n_det : 0u) - 1u)))
        return fail(ctx, GW_EINVAL, "logdet_vjp: det_mask selects no detector of the network");
    if (n == 0) {
        if (mode == MODE_LOGDET) return logdet_zero(ctx, dn.n_det, det_mask, grad_gamma, s);
        if (mode == MODE_SNRGRAD && grad_gamma)
            CK(cudaMemsetAsync(grad_gamma, 0, sizeof(double) * dn.n_det, s));
        return GW_OK;
    }
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure(ctx, ctx->evc, ctx->evc_cap, (size_t)n * EVC))) return st;
    if ((st = ensure(ctx, ctx->sitec, ctx->sitec_cap, (size_t)n * dn.n_site * SC_N))) return st;
    double *xs = nullptr;
    if (fused_grad) {
        if (!grad_snr) return fail(ctx, GW_EINVAL, "fisher: grad_params needs grad_snr");
        if (mixed) {
            if ((st = ensure(ctx, ctx->xsums, ctx->xsums_cap, (size_t)N_SNRGRAD_X * n))) return st;
            xs = ctx->xsums;
        }
        if (!snr) {
            if ((st = ensure(ctx, ctx->snr_tmp, ctx->snr_tmp_cap, (size_t)n))) return st;
            snr = ctx->snr_tmp;
        }
    }
    if (mode == MODE_SNRGRAD && grad_gamma) {
        // per-event terms of the detector-orientation gradient, summed below
        const size_t rows = dn.n_det > N_SNRGRAD_X ? dn.n_det : N_SNRGRAD_X;
        if ((st = ensure(ctx, ctx->xsums, ctx->xsums_cap, rows * n))) return st;
        xs = ctx->xsums;
    }
    if (mixed && (st = ensure(ctx, ctx->sitec_f, ctx->sitec_f_cap, (size_t)n * dn.n_site * SC_N)))
        return st;
    if (mixed && (st = ensure(ctx, ctx->evc_f, ctx->evc_f_cap, (size_t)n * EVC))) return st;
    if ((st = ensure(ctx, ctx->counts, ctx->counts_cap, (size_t)n))) return st;
    if ((st = ensure(ctx, ctx->off, ctx->off_cap, (size_t)n + 1))) return st;
    if ((st = ensure(ctx, ctx->scan, ctx->scan_cap, scan_tmp_size(n)))) return st;
    int32_t *status = status_out;
    if (!status) {
        if ((st = ensure(ctx, ctx->status, ctx->status_cap, (size_t)n))) return st;
        status = ctx->status;
    }
    if (const int64_t nseg = gwi_psd_segments(dn)) {
        if ((st = ensure(ctx, ctx->psd_seg, ctx->psd_seg_cap, (size_t)nseg))) return st;
        if ((st = ensure(ctx, ctx->psd_seg_f, ctx->psd_seg_f_cap, (size_t)2 * nseg))) return st;
        CK(gwi_prep_psd(net, dn, ctx->psd_seg, ctx->psd_seg_f, s));
    }
    const DevCat dc = gwi_dev_cat(cat);
    // the tensor-core Fisher pass (GW_DFLOAT, or GW_FP64 with the tensor-core
    // Gram) takes work items of TC_CHUNK points
    const bool tc = mode == MODE_FISHER && !mixed && fisher_fp64_tc_supported(dn) &&
                    (prec == GW_DFLOAT || ctx->fp64_gram_tc);
    CK(launch_event_setup(dc, dn, np, ctx->evc, ctx->sitec, mixed ? ctx->sitec_f : nullptr,
                          mixed ? ctx->evc_f : nullptr, status, ctx->counts, s,
                          tc ? TC_CHUNK : CHUNK_MAX));
    CK(launch_scan(ctx->counts, n, ctx->off, ctx->scan, s));
    int64_t n_items;
    if (ctx->item_cap > 0) {
        // asynchronous: the kernels take the work count from device memory
        n_items = ctx->item_cap;
        if ((st = ensure(ctx, ctx->partial, ctx->partial_cap, (size_t)n_items * nacc))) return st;
    } else {
        CK(cudaMemcpyAsync(ctx->h_total, ctx->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        n_items = *ctx->h_total;
        if ((st = ensure(ctx, ctx->partial, ctx->partial_cap,
                         (size_t)(n_items > 0 ? n_items : 1) * nacc)))
            return st;
    }
    PointArgs pa;
    pa.net = dn;
    pa.evc = ctx->evc;
    pa.sitec = ctx->sitec;
    pa.sitec_f = ctx->sitec_f;
    pa.evc_f = ctx->evc_f;
    pa.item_off = ctx->off;
    pa.n_ev = n;
    pa.n_items = n_items;
    pa.partial = ctx->partial;
    pa.nacc = nacc;
    pa.cov = cov;
    pa.det_mask = det_mask;
    if (mode == MODE_FISHER) {
        // the tile of this precision and grid-length class (asynchronous mode:
        // the class of the reservation)
        const int cls = ctx->item_cap > 0 ? length_class(ctx->item_cap, ctx->reserved_events)
                                          : length_class(n_items, n);
        const int pi = mixed ? 1 : 0;
        pa.group = ctx->tile_group[pi][cls];
        pa.blocks_per_sm = ctx->tile_bps[pi][cls];
    }
    pa.kerr = ctx->kerr;
    if (ctx->profiling) CK(cudaEventRecord(ctx->ev0, s));
    if (mixed) CK(launch_points_mixed(mode, np, dn.rotation, pa, s));
    else if (tc && prec == GW_DFLOAT) CK(launch_fisher_dfloat_tc(np, dn.rotation, pa, s));
    else if (tc) CK(launch_fisher_fp64_tc(np, dn.rotation, pa, s));
    else CK(launch_points_fp64(mode, np, dn.rotation, pa, s));
    if (ctx->profiling) {
        CK(cudaEventRecord(ctx->ev1, s));
        ctx->ev_recorded = true;
    }
    if (mode == MODE_LOGDET && n_items == 0)
        return logdet_zero(ctx, dn.n_det, det_mask, grad_gamma, s);
    CK(launch_finish(mode, np, dn.n_det, pa, status, snr, snr_det, fisher, grad_snr, grad_params,
                     grad_gamma, xs, s));
    if (fused_grad)
        CK(launch_snr_grad_from_fisher(n, np, mixed, dn.rotation, fisher, snr, xs, ctx->evc,
                                       status, grad_snr, grad_params, s));
    if (mode == MODE_SNRGRAD && grad_gamma) CK(launch_sum_events(xs, n, dn.n_det, grad_gamma, s));
    return GW_OK;
}

}  // namespace

extern "C" {

int gw_abi_version(void) { return 7; }

gw_status gw_create(gw_ctx **out, int device)
{
    if (!out) return GW_EINVAL;
    *out = nullptr;
    gw_ctx *ctx = new (std::nothrow) gw_ctx();
    if (!ctx) return GW_ENOMEM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_total, sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void **)&ctx->kerr, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(ctx->kerr, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->h_total) cudaFreeHost(ctx->h_total);
        if (ctx->kerr) cudaFree(ctx->kerr);
        delete ctx;
        return GW_ECUDA;
    }
    *out = ctx;
    return GW_OK;
}

gw_status gw_destroy(gw_ctx *ctx)
{
    if (!ctx) return GW_OK;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->evc);
    cudaFree(ctx->sitec);
    cudaFree(ctx->sitec_f);
    cudaFree(ctx->evc_f);
    cudaFree(ctx->status);
    cudaFree(ctx->counts);
    cudaFree(ctx->off);
    cudaFree(ctx->scan);
    cudaFree(ctx->partial);
    cudaFree(ctx->xsums);
    cudaFree(ctx->snr_tmp);
    cudaFree(ctx->psd_seg);
    cudaFree(ctx->psd_seg_f);
    cudaFree(ctx->ref_flag);
    cudaFree(ctx->ref_off);
    cudaFree(ctx->ref_scan);
    cudaFree(ctx->ref_pos);
    cudaFree(ctx->ref_rows);
    cudaFree(ctx->ref_F);
    cudaFree(ctx->ref_C);
    cudaFree(ctx->ref_g);
    cudaFree(ctx->ref_v);
    cudaFree(ctx->ref_st);
    cudaFree(ctx->rt_flag);
    cudaFree(ctx->rt_off);
    cudaFree(ctx->rt_scan);
    cudaFree(ctx->rt_pos);
    cudaFree(ctx->rt_rows);
    cudaFree(ctx->rt_F);
    cudaFree(ctx->rt_C);
    cudaFree(ctx->rt_g);
    cudaFree(ctx->rt_v);
    cudaFree(ctx->rt_st);
    cudaFreeHost(ctx->h_total);
    cudaFree(ctx->kerr);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return GW_OK;
}

const char *gw_last_error(const gw_ctx *ctx) { return ctx ? ctx->err : "null context"; }

gw_status gw_reserve(gw_ctx *ctx, int64_t max_events, int64_t max_items, int max_sites)
{
    if (!ctx) return GW_EINVAL;
    if (max_events < 0 || max_items < 0 || max_sites < 0 || max_sites > MAX_SITE)
        return fail(ctx, GW_EINVAL, "reserve: bad sizes");
    CK(cudaSetDevice(ctx->device));
    ctx->item_cap = 0;
    if (max_items == 0) return GW_OK;
    const size_t n = (size_t)(max_events > 0 ? max_events : 1);
    const size_t sites = (size_t)(max_sites > 0 ? max_sites : 1);
    const size_t nacc_max = 1 + 11 * 12 / 2 + N_SNRGRAD_X;
    gw_status st;
    if ((st = ensure(ctx, ctx->evc, ctx->evc_cap, n * EVC))) return st;
    if ((st = ensure(ctx, ctx->evc_f, ctx->evc_f_cap, n * EVC))) return st;
    if ((st = ensure(ctx, ctx->sitec, ctx->sitec_cap, n * sites * SC_N))) return st;
    if ((st = ensure(ctx, ctx->sitec_f, ctx->sitec_f_cap, n * sites * SC_N))) return st;
    if ((st = ensure(ctx, ctx->counts, ctx->counts_cap, n))) return st;
    if ((st = ensure(ctx, ctx->off, ctx->off_cap, n + 1))) return st;
    if ((st = ensure(ctx, ctx->scan, ctx->scan_cap, scan_tmp_size((int64_t)n)))) return st;
    if ((st = ensure(ctx, ctx->status, ctx->status_cap, n))) return st;
    if ((st = ensure(ctx, ctx->xsums, ctx->xsums_cap, (size_t)N_SNRGRAD_X * n))) return st;
    if ((st = ensure(ctx, ctx->snr_tmp, ctx->snr_tmp_cap, n))) return st;
    if ((st = ensure(ctx, ctx->partial, ctx->partial_cap, (size_t)max_items * nacc_max))) return st;
    ctx->item_cap = max_items;
    ctx->reserved_events = (int64_t)n;
    return GW_OK;
}

gw_status gw_set_tile(gw_ctx *ctx, gw_precision prec, int length_class_, int group,
                      int blocks_per_sm)
{
    if (!ctx) return GW_EINVAL;
    if ((prec != GW_FP64 && prec != GW_MIXED) || length_class_ < 0 || length_class_ > 2 ||
        (group != 4 && group != 8 && group != 16) || (blocks_per_sm != 1 && blocks_per_sm != 2))
        return fail(ctx, GW_EINVAL, "set_tile: precision 0/1, class 0..2, group 4/8/16, "
                    "blocks per SM 1/2");
    ctx->tile_group[prec][length_class_] = group;
    ctx->tile_bps[prec][length_class_] = blocks_per_sm;
    return GW_OK;
}

gw_status gw_set_fp64_gram(gw_ctx *ctx, int tensor)
{
    if (!ctx) return GW_EINVAL;
    if (tensor != 0 && tensor != 1) return fail(ctx, GW_EINVAL, "set_fp64_gram: 0 or 1");
    ctx->fp64_gram_tc = tensor;
    return GW_OK;
}

gw_status gw_kernel_faults(gw_ctx *ctx, int32_t *faults, int reset)
{
    if (!ctx || !faults) return GW_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpy(faults, ctx->kerr, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (reset) CK(cudaMemset(ctx->kerr, 0, sizeof(int32_t)));
    return GW_OK;
}

gw_status gw_autotune(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                      gw_precision prec, int n_par, int reps, int32_t *length_class_out,
                      int32_t *group_out, int32_t *bps_out, double *ms_out, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat || cat->n <= 0 || reps < 1 || reps > 100)
        return fail(ctx, GW_EINVAL, "autotune: a non-empty catalog and 1 <= reps <= 100");
    if (prec != GW_FP64 && prec != GW_MIXED) return fail(ctx, GW_EINVAL, "bad precision");
    if (ctx->item_cap > 0) return fail(ctx, GW_EINVAL, "autotune: release gw_reserve first");
    const int64_t n = cat->n;
    const int npk = n_par * (n_par + 1) / 2;
    gw_status st;
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure(ctx, ctx->ref_F, ctx->ref_F_cap, (size_t)npk * n))) return st;
    if ((st = ensure(ctx, ctx->ref_v, ctx->ref_v_cap, (size_t)4 * n))) return st;
    if ((st = ensure(ctx, ctx->ref_st, ctx->ref_st_cap, (size_t)2 * n))) return st;
    // one pass for the work count (the grid-length class) and the workspace
    if ((st = run_points(ctx, cat, net, prec, MODE_FISHER, n_par, ctx->ref_st, ctx->ref_v,
                         nullptr, ctx->ref_F, nullptr, nullptr, nullptr, nullptr, stream)))
        return st;
    const int cls = length_class(*ctx->h_total, n);
    const int pi = prec == GW_MIXED ? 1 : 0;
    const int old_g = ctx->tile_group[pi][cls], old_b = ctx->tile_bps[pi][cls];
    const int old_prof = ctx->profiling;
    if ((st = gw_set_profiling(ctx, 1))) return st;
    static const int G[3] = {4, 8, 16};
    double best = 1e300;
    int bg = old_g, bb = old_b;
    for (int gi = 0; gi < 3; gi++)
        for (int b = 1; b <= 2; b++) {
            ctx->tile_group[pi][cls] = G[gi];
            ctx->tile_bps[pi][cls] = b;
            double tmin = 1e300;
            for (int r = 0; r < reps + 1; r++) {   // the first run is a warm-up
                if ((st = run_points(ctx, cat, net, prec, MODE_FISHER, n_par, ctx->ref_st,
                                     ctx->ref_v, nullptr, ctx->ref_F, nullptr, nullptr, nullptr,
                                     nullptr, stream)))
                    return st;
                const double ms = gw_point_kernel_ms(ctx);
                if (r > 0 && ms >= 0.0 && ms < tmin) tmin = ms;
            }
            if (ms_out) ms_out[gi * 2 + (b - 1)] = tmin;
            if (tmin < best) {
                best = tmin;
                bg = G[gi];
                bb = b;
            }
        }
    gw_set_profiling(ctx, old_prof);
    ctx->tile_group[pi][cls] = bg;
    ctx->tile_bps[pi][cls] = bb;
    if (length_class_out) *length_class_out = cls;
    if (group_out) *group_out = bg;
    if (bps_out) *bps_out = bb;
    return GW_OK;
}

gw_status gw_set_profiling(gw_ctx *ctx, int enable)
{
    if (!ctx) return GW_EINVAL;
    CK(cudaSetDevice(ctx->device));
    if (enable && !ctx->ev0) {
        CK(cudaEventCreate(&ctx->ev0));
        CK(cudaEventCreate(&ctx->ev1));
    }
    ctx->profiling = enable ? 1 : 0;
    ctx->ev_recorded = false;
    return GW_OK;
}

double gw_point_kernel_ms(gw_ctx *ctx)
{
    if (!ctx || !ctx->ev_recorded) return -1.0;
    float ms = -1.0f;
    if (cudaEventSynchronize(ctx->ev1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    return (double)ms;
}

gw_status gw_prepare_catalog(gw_ctx *ctx, int64_t n, const double *m1, const double *m2,
                             const double *chi1, const double *chi2, const double *lam1,
                             const double *lam2, const double *dL_Mpc, const uint8_t *zflag,
                             const double *tcoal, const double *fmin, const int32_t *npts_given,
                             int32_t npts_fixed, double per_efold, int32_t npts_lo,
                             int32_t npts_hi, double *Mc, double *eta, double *dL_Gpc,
                             double *chi1o, double *chi2o, double *LamT, double *dLamT,
                             double *tc_s, double *fmax, int32_t *npts, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0) return fail(ctx, GW_EINVAL, "n < 0");
    if (n == 0) return GW_OK;
    if (!m1 || !m2 || !chi1 || !chi2 || !dL_Mpc || !zflag || !tcoal || !fmin || !Mc || !eta ||
        !dL_Gpc || !chi1o || !chi2o || !LamT || !dLamT || !tc_s || !fmax || !npts)
        return fail(ctx, GW_EINVAL, "prepare: a required array is null");
    if (!npts_given && npts_fixed <= 0 && !(per_efold > 0 && npts_lo >= 2 && npts_hi >= npts_lo))
        return fail(ctx, GW_EINVAL, "prepare: no valid grid-length rule");
    CK(cudaSetDevice(ctx->device));
    CK(launch_prepare(n, m1, m2, chi1, chi2, lam1, lam2, dL_Mpc, zflag, tcoal, fmin, npts_given,
                      npts_fixed, per_efold, npts_lo, npts_hi, Mc, eta, dL_Gpc, chi1o, chi2o, LamT,
                      dLamT, tc_s, fmax, npts, (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_snr(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                 double *snr, double *snr_det, int32_t *status, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (!snr && cat->n > 0) return fail(ctx, GW_EINVAL, "snr: output is null");
    // the parameter set does not matter for the SNR: run as 9-parameter events
    // with a catalog view whose pset is ignored
    gw_catalog c9 = *cat;
    c9.pset = nullptr;
    return run_points(ctx, &c9, net, prec, MODE_SNR, 9, status, snr, snr_det, nullptr, nullptr,
                      nullptr, nullptr, nullptr, stream);
}

gw_status gw_select_snr(gw_ctx *ctx, const double *snr, int64_t n, double threshold,
                        int64_t *sel, int64_t *n_sel, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || !n_sel) return fail(ctx, GW_EINVAL, "select: n < 0 or n_sel null");
    *n_sel = 0;
    if (n == 0) return GW_OK;
    if (!snr || !sel) return fail(ctx, GW_EINVAL, "select: null array");
    if (std::isnan(threshold)) return fail(ctx, GW_EINVAL, "select: threshold is NaN");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    gw_status st;
    if ((st = ensure(ctx, ctx->counts, ctx->counts_cap, (size_t)n))) return st;
    if ((st = ensure(ctx, ctx->off, ctx->off_cap, (size_t)n + 1))) return st;
    if ((st = ensure(ctx, ctx->scan, ctx->scan_cap, scan_tmp_size(n)))) return st;
    CK(launch_select(snr, n, threshold, ctx->counts, ctx->off, ctx->scan, sel, s));
    CK(cudaMemcpyAsync(n_sel, ctx->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return GW_OK;
}

namespace {
// kept parameter slots of a keep mask over n_par parameters (0 = all)
int kept_slots(uint32_t keep, int n_par, int *idx)
{
    if (keep == 0) keep = (1u << n_par) - 1u;
    int k = 0;
    for (int i = 0; i < n_par; i++)
        if ((keep >> i) & 1u) idx[k++] = i;
    return (keep >> n_par) ? -1 : k;
}
}  // namespace

gw_status gw_fisher_eig(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, int normalize,
                        double *eigval, double *eigvec, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || n_par < 1 || n_par > 11) return fail(ctx, GW_EINVAL, "eig: bad n or n_par");
    if (n == 0) return GW_OK;
    if (!fisher || (!eigval && !eigvec)) return fail(ctx, GW_EINVAL, "eig: null array");
    CK(cudaSetDevice(ctx->device));
    CK(launch_fisher_eig(n, n_par, normalize, fisher, eigval, eigvec, (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_covariance(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, uint32_t keep,
                        const double *prior, int method, double thresh, double cond_max,
                        double *cov, double *cond, double *inv_err, int32_t *status,
                        void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || n_par < 1 || n_par > 11) return fail(ctx, GW_EINVAL, "covariance: bad n or n_par");
    if (method < GW_INV_CHO || method > GW_INV_LU)
        return fail(ctx, GW_EINVAL, "covariance: unknown method %d", method);
    if (!(thresh >= 0.0) || !(thresh < 1.0))
        return fail(ctx, GW_EINVAL, "covariance: thresh must be in [0, 1)");
    CovArgs a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.P = n_par;
    a.Pk = kept_slots(keep, n_par, a.idx);
    if (a.Pk < 1) return fail(ctx, GW_EINVAL, "covariance: keep mask 0x%x for %d parameters", keep, n_par);
    if (prior)
        for (int i = 0; i < n_par; i++) {
            if (!std::isfinite(prior[i]) || prior[i] < 0.0)
                return fail(ctx, GW_EINVAL, "covariance: prior[%d] must be finite and >= 0", i);
            a.prior[i] = prior[i];
        }
    a.method = method;
    a.thresh = thresh;
    a.cond_max = std::isnan(cond_max) ? INFINITY : cond_max;
    if (n == 0) return GW_OK;
    if (!fisher || !cov) return fail(ctx, GW_EINVAL, "covariance: null array");
    CK(cudaSetDevice(ctx->device));
    CK(launch_covariance(a, fisher, cov, cond, inv_err, status, (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_packed_submatrix(gw_ctx *ctx, const double *in, int64_t n, int n_par, uint32_t keep,
                              double *out, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || n_par < 1 || n_par > 11) return fail(ctx, GW_EINVAL, "submatrix: bad n or n_par");
    SubIdx si;
    const int K = kept_slots(keep, n_par, si.idx);
    if (K < 1) return fail(ctx, GW_EINVAL, "submatrix: keep mask 0x%x for %d parameters", keep, n_par);
    if (n == 0) return GW_OK;
    if (!in || !out) return fail(ctx, GW_EINVAL, "submatrix: null array");
    CK(cudaSetDevice(ctx->device));
    CK(launch_submatrix(n, n_par, K, si, in, out, (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_perturb_fisher(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, double eps,
                            const double *r, double *out, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || n_par < 1 || n_par > 11 || !std::isfinite(eps))
        return fail(ctx, GW_EINVAL, "perturb: bad n, n_par or eps");
    if (n == 0) return GW_OK;
    if (!fisher || !r || !out) return fail(ctx, GW_EINVAL, "perturb: null array");
    CK(cudaSetDevice(ctx->device));
    CK(launch_perturb(n * (int64_t)(n_par * (n_par + 1) / 2), eps, fisher, r, out,
                      (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_sky_area(gw_ctx *ctx, const double *cov, int64_t n, int n_par, int i_theta,
                      int i_phi, const double *theta, double perc, int units, double *area,
                      void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || n_par < 2 || n_par > 11 || i_theta < 0 || i_theta >= n_par || i_phi < 0 ||
        i_phi >= n_par || i_theta == i_phi)
        return fail(ctx, GW_EINVAL, "sky_area: bad n, n_par or parameter slots");
    if (!(perc > 0.0) || !(perc < 100.0) || (units != 0 && units != 1))
        return fail(ctx, GW_EINVAL, "sky_area: perc must be in (0, 100), units 0 or 1");
    if (n == 0) return GW_OK;
    if (!cov || !theta || !area) return fail(ctx, GW_EINVAL, "sky_area: null array");
    CK(cudaSetDevice(ctx->device));
    CK(launch_sky_area(n, n_par, i_theta, i_phi, cov, theta, perc, units, area,
                       (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_strain(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                    int64_t total_points, double *re, double *im, double *freq,
                    int64_t *point_off, int32_t *status_out, void *stream)
{
    if (!ctx) return GW_EINVAL;
    gw_status st = gwi_check_cat(ctx, cat, 9);
    if (st) return st;
    if (prec != GW_FP64 && prec != GW_MIXED && prec != GW_DFLOAT)
        return fail(ctx, GW_EINVAL, "strain: precision");
    DevNet dn;
    if ((st = gwi_build_net(ctx, net, dn))) return st;
    const int64_t n = cat->n;
    if (n == 0) return total_points == 0 ? GW_OK : fail(ctx, GW_EINVAL, "strain: total_points != 0");
    if (!re || !im) return fail(ctx, GW_EINVAL, "strain: null output");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    if ((st = ensure(ctx, ctx->evc, ctx->evc_cap, (size_t)n * EVC))) return st;
    if ((st = ensure(ctx, ctx->sitec, ctx->sitec_cap, (size_t)n * dn.n_site * SC_N))) return st;
    if ((st = ensure(ctx, ctx->counts, ctx->counts_cap, (size_t)n))) return st;
    if ((st = ensure(ctx, ctx->off, ctx->off_cap, (size_t)n + 1))) return st;
    if ((st = ensure(ctx, ctx->scan, ctx->scan_cap, scan_tmp_size(n)))) return st;
    int32_t *status = status_out;
    if (!status) {
        if ((st = ensure(ctx, ctx->status, ctx->status_cap, (size_t)n))) return st;
        status = ctx->status;
    }
    int64_t *poff = point_off ? point_off : ctx->off;
    CK(launch_point_offsets(cat->npts, cat->sel, n, ctx->counts, poff, ctx->scan, s));
    int64_t tot = 0;
    CK(cudaMemcpyAsync(&tot, poff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (tot != total_points)
        return fail(ctx, GW_EINVAL, "strain: total_points %lld, the grids hold %lld points",
                    (long long)total_points, (long long)tot);
    // the per-event constants of the Fisher pass (parameter set ignored)
    gw_catalog c9 = *cat;
    c9.pset = nullptr;
    const DevCat dc = gwi_dev_cat(&c9);
    CK(launch_event_setup(dc, dn, 9, ctx->evc, ctx->sitec, nullptr, nullptr, status, ctx->counts, s));
    CK(launch_strain(dn, n, total_points, prec == GW_MIXED ? 1 : 0, ctx->evc, ctx->sitec, status,
                     poff, re, im, freq, s));
    return GW_OK;
}

gw_status gw_fisher(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                    int n_par, double *fisher, double *snr, int32_t *status,
                    const double *grad_snr, double *grad_params, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (!fisher && cat->n > 0) return fail(ctx, GW_EINVAL, "fisher: output is null");
    return run_points(ctx, cat, net, prec, MODE_FISHER, n_par, status, snr, nullptr, fisher,
                      grad_snr, grad_params, nullptr, nullptr, stream);
}

// the refinement with the recomputing pass's precision as a parameter:
// gw_fisher_refine recomputes in FP64, gw_fisher_routed in double-float
static gw_status refine_with(gw_precision rprec, gw_ctx *ctx, const gw_catalog *cat,
                             const gw_network *net, int n_par, double cond_th, double cond_max,
                             double *fisher, double *snr, int32_t *status, const double *grad_snr,
                             double *grad_params, double *cov, double *cond, double *inv_err,
                             int32_t *inv_status, uint8_t *refined, int64_t *n_refined,
                             void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n_refined) *n_refined = 0;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (n_par != 9 && n_par != 11) return fail(ctx, GW_EINVAL, "n_par must be 9 or 11");
    if (std::isnan(cond_th)) return fail(ctx, GW_EINVAL, "refine: cond_th is NaN");
    const int64_t n = cat->n;
    if (n == 0) return GW_OK;
    if (!fisher || !status || !cov || !cond || !inv_status)
        return fail(ctx, GW_EINVAL, "refine: fisher, status, cov, cond and inv_status are required");
    if ((grad_params != nullptr) != (grad_snr != nullptr))
        return fail(ctx, GW_EINVAL, "refine: grad_params and grad_snr go together");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    gw_status st;
    if ((st = ensure(ctx, ctx->ref_flag, ctx->ref_flag_cap, (size_t)n))) return st;
    if ((st = ensure(ctx, ctx->ref_off, ctx->ref_off_cap, (size_t)n + 1))) return st;
    if ((st = ensure(ctx, ctx->ref_scan, ctx->ref_scan_cap, scan_tmp_size(n)))) return st;
    if ((st = ensure(ctx, ctx->ref_pos, ctx->ref_pos_cap, (size_t)n))) return st;
    if ((st = ensure(ctx, ctx->ref_rows, ctx->ref_rows_cap, (size_t)n))) return st;
    CK(launch_refine_select(n, cond_th, status, inv_status, cond, cat->sel, ctx->ref_flag,
                            ctx->ref_off, ctx->ref_scan, ctx->ref_pos, ctx->ref_rows, refined, s));
    CK(cudaMemcpyAsync(ctx->h_total, ctx->ref_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t m = *ctx->h_total;
    if (n_refined) *n_refined = m;
    if (m == 0) return GW_OK;
    const int npk = n_par * (n_par + 1) / 2;
    if ((st = ensure(ctx, ctx->ref_F, ctx->ref_F_cap, (size_t)npk * m))) return st;
    if ((st = ensure(ctx, ctx->ref_C, ctx->ref_C_cap, (size_t)npk * m))) return st;
    if ((st = ensure(ctx, ctx->ref_g, ctx->ref_g_cap, (size_t)n_par * m))) return st;
    if ((st = ensure(ctx, ctx->ref_v, ctx->ref_v_cap, (size_t)4 * m))) return st;
    if ((st = ensure(ctx, ctx->ref_st, ctx->ref_st_cap, (size_t)2 * m))) return st;
    double *r_snr = ctx->ref_v, *r_gin = ctx->ref_v + m, *r_cond = ctx->ref_v + 2 * m,
           *r_err = ctx->ref_v + 3 * m;
    int32_t *r_st = ctx->ref_st, *r_sti = ctx->ref_st + m;
    // the flagged events as a catalog of their own (rows through the call's
    // selection), FP64 Fisher pass and inversion
    gw_catalog sub = *cat;
    sub.n = m;
    sub.sel = ctx->ref_rows;
    if (grad_snr) CK(launch_gather(m, ctx->ref_pos, grad_snr, r_gin, s));
    if ((st = run_points(ctx, &sub, net, rprec, MODE_FISHER, n_par, r_st, r_snr, nullptr,
                         ctx->ref_F, grad_snr ? r_gin : nullptr, grad_snr ? ctx->ref_g : nullptr,
                         nullptr, nullptr, stream)))
        return st;
    CK(launch_invert(ctx->ref_F, m, n_par, cond_max, ctx->ref_C, r_cond, r_err, r_sti, s));
    // written back in place, at the call's indices of the flagged events
    const int64_t *pos = ctx->ref_pos;
    ScatterSet set;
    set.add(ctx->ref_F, fisher, npk, 8);
    set.add(ctx->ref_C, cov, npk, 8);
    set.add(r_snr, snr, 1, 8);
    set.add(r_cond, cond, 1, 8);
    set.add(r_err, inv_err, 1, 8);
    if (grad_params) set.add(ctx->ref_g, grad_params, n_par, 8);
    set.add(r_st, status, 1, 4);
    set.add(r_sti, inv_status, 1, 4);
    CK(launch_scatter_set(m, n, pos, set, s));
    return GW_OK;
}

gw_status gw_fisher_refine(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, int n_par,
                           double cond_th, double cond_max, double *fisher, double *snr,
                           int32_t *status, const double *grad_snr, double *grad_params,
                           double *cov, double *cond, double *inv_err, int32_t *inv_status,
                           uint8_t *refined, int64_t *n_refined, void *stream)
{
    return refine_with(GW_FP64, ctx, cat, net, n_par, cond_th, cond_max, fisher, snr, status,
                       grad_snr, grad_params, cov, cond, inv_err, inv_status, refined, n_refined,
                       stream);
}

gw_status gw_fisher_routed(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, int n_par,
                           uint32_t dfloat_psets, double cond_th, double cond_max, double *fisher,
                           double *snr, int32_t *status, const double *grad_snr,
                           double *grad_params, double *cov, double *cond, double *inv_err,
                           int32_t *inv_status, int64_t *n_dfloat, int64_t *n_refined,
                           void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n_dfloat) *n_dfloat = 0;
    if (n_refined) *n_refined = 0;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (n_par != 9 && n_par != 11) return fail(ctx, GW_EINVAL, "n_par must be 9 or 11");
    if (std::isnan(cond_th)) return fail(ctx, GW_EINVAL, "routed: cond_th is NaN");
    const int64_t n = cat->n;
    if (n == 0) return GW_OK;
    if (!fisher || !status || !cov || !cond || !inv_status)
        return fail(ctx, GW_EINVAL, "routed: fisher, status, cov, cond and inv_status are required");
    if ((grad_params != nullptr) != (grad_snr != nullptr))
        return fail(ctx, GW_EINVAL, "routed: grad_params and grad_snr go together");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    gw_status st;
    if ((st = ensure(ctx, ctx->rt_flag, ctx->rt_flag_cap, (size_t)2 * n))) return st;
    if ((st = ensure(ctx, ctx->rt_off, ctx->rt_off_cap, (size_t)2 * n + 2))) return st;
    if ((st = ensure(ctx, ctx->rt_scan, ctx->rt_scan_cap, scan_tmp_size(n)))) return st;
    if ((st = ensure(ctx, ctx->rt_pos, ctx->rt_pos_cap, (size_t)2 * n))) return st;
    if ((st = ensure(ctx, ctx->rt_rows, ctx->rt_rows_cap, (size_t)2 * n))) return st;
    CK(launch_split_pset(n, cat->pset, cat->sel, dfloat_psets, ctx->rt_flag, ctx->rt_off,
                         ctx->rt_scan, ctx->rt_pos, ctx->rt_rows, s));
    CK(cudaMemcpyAsync(ctx->h_total, ctx->rt_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int64_t m_df = *ctx->h_total, m_mx = n - m_df;
    if (n_dfloat) *n_dfloat = m_df;
    const int npk = n_par * (n_par + 1) / 2;
    if ((st = ensure(ctx, ctx->rt_F, ctx->rt_F_cap, (size_t)npk * n))) return st;
    if ((st = ensure(ctx, ctx->rt_C, ctx->rt_C_cap, (size_t)npk * n))) return st;
    if (grad_snr && (st = ensure(ctx, ctx->rt_g, ctx->rt_g_cap, (size_t)n_par * n))) return st;
    if ((st = ensure(ctx, ctx->rt_v, ctx->rt_v_cap, (size_t)4 * n))) return st;
    if ((st = ensure(ctx, ctx->rt_st, ctx->rt_st_cap, (size_t)2 * n))) return st;
    // part b (the mixed events) first: its Fisher pass and inversion, its
    // results written to the call's outputs, and the events that fail the
    // conditioning check marked for part a; then part a (the double-float
    // events and the marked ones) in one pass, written over them.  Each
    // part's results are event-minor in the temporaries, from offset 0.
    auto run_part = [&](gw_precision prec, int64_t m, const int64_t *pos,
                        const int64_t *rows) -> gw_status {
        gw_catalog sub = *cat;
        sub.n = m;
        sub.sel = rows;
        double *F = ctx->rt_F, *C = ctx->rt_C;
        double *g = grad_snr ? ctx->rt_g : nullptr;
        double *v_snr = ctx->rt_v, *v_gin = ctx->rt_v + n, *v_cond = ctx->rt_v + 2 * n,
               *v_err = ctx->rt_v + 3 * n;
        int32_t *v_st = ctx->rt_st, *v_sti = ctx->rt_st + n;
        gw_status e;
        if (grad_snr) CK(launch_gather(m, pos, grad_snr, v_gin, s));
        if ((e = run_points(ctx, &sub, net, prec, MODE_FISHER, n_par, v_st, v_snr, nullptr, F,
                            grad_snr ? v_gin : nullptr, g, nullptr, nullptr, stream)))
            return e;
        CK(launch_invert(F, m, n_par, cond_max, C, v_cond, v_err, v_sti, s));
        if (prec == GW_MIXED)
            CK(launch_route_recompute(m, cond_th, v_st, v_sti, v_cond, pos, n, cat->sel,
                                      ctx->rt_flag, ctx->rt_off, ctx->rt_scan, ctx->rt_pos,
                                      ctx->rt_rows, s));
        ScatterSet set;
        set.add(F, fisher, npk, 8);
        set.add(C, cov, npk, 8);
        set.add(v_snr, snr, 1, 8);
        set.add(v_cond, cond, 1, 8);
        set.add(v_err, inv_err, 1, 8);
        if (grad_params) set.add(g, grad_params, n_par, 8);
        set.add(v_st, status, 1, 4);
        set.add(v_sti, inv_status, 1, 4);
        CK(launch_scatter_set(m, n, pos, set, s));
        return GW_OK;
    };
    int64_t m_a = m_df;
    if (m_mx > 0) {
        if ((st = run_part(GW_MIXED, m_mx, ctx->rt_pos + n, ctx->rt_rows + n))) return st;
        CK(cudaMemcpyAsync(ctx->h_total, ctx->rt_off + n, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        m_a = *ctx->h_total;
        if (n_refined) *n_refined = m_a - m_df;
    }
    if (m_a > 0 && (st = run_part(GW_DFLOAT, m_a, ctx->rt_pos, ctx->rt_rows))) return st;
    return GW_OK;
}

gw_status gw_fisher_inverse(gw_ctx *ctx, const double *fisher, int64_t n, int n_par,
                            double cond_max, double *cov, double *cond, double *inv_err,
                            int32_t *status, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (n < 0 || (n > 0 && (!fisher || !cov)))
        return fail(ctx, GW_EINVAL, "fisher_inverse: bad arguments");
    if (n_par != 9 && n_par != 11) return fail(ctx, GW_EINVAL, "n_par must be 9 or 11");
    if (n == 0) return GW_OK;
    CK(cudaSetDevice(ctx->device));
    int32_t *st = status;
    if (!st) {
        gw_status e = ensure(ctx, ctx->status, ctx->status_cap, (size_t)n);
        if (e) return e;
        st = ctx->status;
    }
    CK(launch_invert(fisher, n, n_par, cond_max, cov, cond, inv_err, st, (cudaStream_t)stream));
    return GW_OK;
}

gw_status gw_snr_vjp(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                     int n_par, const double *grad_snr, double *grad_params, double *grad_gamma,
                     void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if ((!grad_snr || !grad_params) && cat->n > 0)
        return fail(ctx, GW_EINVAL, "snr_vjp: null array");
    return run_points(ctx, cat, net, prec, MODE_SNRGRAD, n_par, nullptr, nullptr, nullptr,
                      nullptr, grad_snr, grad_params, nullptr, grad_gamma, stream);
}

gw_status gw_logdet_vjp_detangles(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                                  gw_precision prec, int n_par, const double *cov,
                                  double *grad_gamma, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (!grad_gamma || (!cov && cat->n > 0)) return fail(ctx, GW_EINVAL, "logdet_vjp: null array");
    return run_points(ctx, cat, net, prec, MODE_LOGDET, n_par, nullptr, nullptr, nullptr,
                      nullptr, nullptr, nullptr, cov, grad_gamma, stream);
}

gw_status gw_logdet_vjp_detangles_masked(gw_ctx *ctx, const gw_catalog *cat,
                                         const gw_network *net, gw_precision prec, int n_par,
                                         const double *cov, uint32_t det_mask,
                                         double *grad_gamma, void *stream)
{
    if (!ctx) return GW_EINVAL;
    if (!cat) return fail(ctx, GW_EINVAL, "catalog: null");
    if (!grad_gamma || (!cov && cat->n > 0)) return fail(ctx, GW_EINVAL, "logdet_vjp: null array");
    return run_points(ctx, cat, net, prec, MODE_LOGDET, n_par, nullptr, nullptr, nullptr,
                      nullptr, nullptr, nullptr, cov, grad_gamma, stream, det_mask);
}

}  // extern "C"
