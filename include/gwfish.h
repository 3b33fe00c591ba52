/*
 * gwfish.h -- C ABI of the GB300 Fisher-forecast library (libgwfish.so).
 *
 * The library evaluates, for every event of a catalog of compact-binary
 * coalescences, the hot path of the Fisher-information forecast of GWFAST
 * (arXiv:2207.06910): the TaylorF2 waveform on a per-event log frequency grid,
 * projected on a network of L-shaped and triangular interferometers with Earth
 * rotation, its derivatives with respect to the 9 or 11 source parameters, the
 * network SNR (Sec. 3.2, Eqs. 3.1-3.2) and Fisher matrix (Sec. 3.2, Eq. 3.3),
 * the Cholesky-based covariance with a conditioning check (Sec. 4.1), and
 * vector-Jacobian products of the SNR and of sum_e log det Gamma_e.
 *
 * General rules for every entry point
 *  - Array arguments marked DEVICE are device pointers (cudaMalloc / PyTorch
 *    CUDA tensors) on the context's device; HOST marks host pointers.  The
 *    caller owns all of them; the library never frees caller memory.
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and is asynchronous unless stated otherwise.  gw_snr, gw_fisher
 *    and the VJPs read back one 8-byte work count per call (a synchronisation
 *    of `stream`); gw_fisher_inverse and gw_prepare_catalog do not synchronise.
 *  - The return value reports argument and launch errors only (GW_EINVAL,
 *    GW_ECUDA, GW_ENOMEM).  Per-event numerical problems are reported in the
 *    per-event `status` bitfield (GW_ST_*) and their outputs are NaN.
 *  - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef GWFISH_H
#define GWFISH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GW_OK = 0,
    GW_EINVAL = 1,       /* bad argument (null pointer, size, network table) */
    GW_ECUDA = 2,        /* a CUDA call failed; gw_last_error() has the text  */
    GW_ENOMEM = 3,       /* workspace allocation failed                       */
    GW_EUNSUPPORTED = 4, /* valid request this build does not implement       */
    GW_ETOOLARGE = 5     /* request exceeds a fixed capacity (gw_fisher_noalloc) */
} gw_status;

typedef enum {
    GW_FP64 = 0,   /* every operation in FP64                                  */
    GW_MIXED = 1   /* FP64 grid, phase derivatives, tau*, Earth angle and
                      accumulation; FP32 amplitude, patterns, tangents and
                      products with exactly compensated (double-float) sums  */
} gw_precision;

/* per-event status bits */
enum {
    GW_ST_NOT_PD = 1,       /* Cholesky pivot <= 0                             */
    GW_ST_COND_GT_MAX = 2,  /* condition number above cond_max: not inverted   */
    GW_ST_NONFINITE = 4,    /* NaN / Inf in the input matrix                   */
    GW_ST_EMPTY_GRID = 8,   /* fmax <= fmin or npts < 2                        */
    GW_ST_BAD_PARAM = 16,   /* Mc <= 0, eta outside (0, 1/4], dL <= 0, wrong
                               parameter set for n_par                         */
    GW_ST_ILL_COND = 32,    /* condition number above 1/DBL_EPSILON (Sec. 4:
                               inversion unreliable beyond inverse precision)  */
    GW_ST_OVERFLOW = 64     /* work items beyond the gw_reserve capacity       */
};

/* A work item is a run of at most GW_ITEM_POINTS consecutive grid points of one
 * event: an event of npts points has ceil(npts / GW_ITEM_POINTS) items. */
#define GW_ITEM_POINTS 256

/* Fisher parameter order (the fixed order of Sec. 3.2): slot 0..8 =
 *   Mc [Msun, detector frame], eta, dL [Gpc], theta, phi, iota, psi [rad],
 *   tc [s], Phic [rad];
 * slots 9, 10 depend on the event's parameter set:
 *   pset 1 -> chi1z, chi2z;  pset 2 -> LambdaTilde, deltaLambdaTilde.
 * pset 0 events have 9 parameters. */

/* Catalog: structure of arrays, every pointer DEVICE, length n, read only. */
typedef struct gw_catalog {
    int64_t n;
    const double *Mc, *eta, *dL, *theta, *phi, *iota, *psi, *tc, *Phic;
    const double *chi1z, *chi2z;      /* NULL -> 0 (spins enter the phase)    */
    const double *LamT, *dLamT;       /* NULL -> 0 (tidal phase)              */
    const int8_t *pset;               /* 0, 1 or 2 (see above)                */
    const double *fmin, *fmax;        /* grid ends [Hz]                       */
    const int32_t *npts;              /* grid points, log spaced (Sec. 2.2)   */
} gw_catalog;

/* Interferometer.  shape 0: L-shaped with opening angle zeta and bisector at
 * gamma counter-clockwise from local East; shape 1: triangle of three
 * co-located 60-degree interferometers (zeta ignored) whose bisectors are at
 * gamma + 30 deg + 120 deg k (Table 2: gamma of a triangle is its first arm).
 * Angles in radians.  psd indexes the network's PSD table. */
typedef struct gw_detector {
    double lat, lon, gamma, zeta;
    int32_t shape, psd;
} gw_detector;

/* Noise PSD: S_n(f) = scale * sum_{j<nterm} coef[j] (f/f0)^pw[j], nterm <= 4. */
typedef struct gw_psd {
    double f0, scale;
    int32_t nterm, reserved;
    double coef[4], pw[4];
} gw_psd;

/* Network (HOST memory, read during the call only).  n_det <= 8 with at most
 * 8 distinct sites, n_psd <= 4.  earth_rotation 0 evaluates the patterns and
 * the Doppler phase at the Earth angle of the event's tc and holds them fixed
 * (not differentiated); 1 follows t(f) = tc - tau*(f). */
typedef struct gw_network {
    int32_t n_det, earth_rotation;
    const gw_detector *det;
    int32_t n_psd, reserved;
    const gw_psd *psd;
} gw_network;

typedef struct gw_ctx gw_ctx;

/* Create a context on CUDA device `device`; it owns the workspace (grown on
 * demand, freed by gw_destroy).  *ctx is NULL on failure. */
gw_status gw_create(gw_ctx **ctx, int device);
gw_status gw_destroy(gw_ctx *ctx);
/* Text of the last error on this context (static storage, never NULL). */
const char *gw_last_error(const gw_ctx *ctx);
/* ABI version of this header (incremented on any signature change): 2. */
int gw_abi_version(void);

/* Reserve workspace for up to max_events events on up to max_sites detector
 * sites and max_items work items, and switch the context to asynchronous mode:
 * gw_snr, gw_fisher, gw_snr_vjp and gw_logdet_vjp_detangles then neither read
 * the work count back (no synchronisation) nor allocate while a call fits the
 * reservation, so a sequence of calls can be captured in a CUDA graph and
 * replayed.  The kernels take the work count from device memory; events whose
 * work items fall beyond max_items get GW_ST_OVERFLOW and NaN outputs.  A call
 * that needs more events or sites than reserved grows the workspace (which is
 * not allowed during capture and then fails with GW_ECUDA).  max_items = 0
 * returns to the synchronous default.  No counterpart in the paper. */
gw_status gw_reserve(gw_ctx *ctx, int64_t max_events, int64_t max_items, int max_sites);

/* Measurement hook (no counterpart in the paper): when enabled, the context
 * records CUDA events on the call's stream around every point-loop kernel
 * launch (the fused SNR / Fisher / VJP kernel).  gw_point_kernel_ms waits for
 * the last recorded pair and returns its duration in milliseconds (negative
 * when nothing was recorded). */
gw_status gw_set_profiling(gw_ctx *ctx, int enable);
double gw_point_kernel_ms(gw_ctx *ctx);

/* Catalog preparation (Sec. 2.1; Eq. 2.2; f_ISCO of the Sec. 2.2 footnote).
 * DEVICE inputs, length n: m1, m2 [Msun], chi1, chi2, lam1, lam2 (NULL -> 0),
 * dL_Mpc, zflag (1: masses are source frame, multiplied by 1+z with
 * z = H0 dL / c, H0 = 70 km/s/Mpc), tcoal [sidereal days], fmin [Hz].
 * Grid length: npts_given (DEVICE, may be NULL) if non-NULL, else
 * npts_fixed if > 0, else clamp(ceil(per_efold ln(f_ISCO/fmin)), lo, hi).
 * DEVICE outputs, length n: Mc [Msun], eta, dL_Gpc, chi1o, chi2o (swapped with
 * the masses so that m1 >= m2), LamT, dLamT, tc_s, fmax (= f_ISCO), npts. */
gw_status gw_prepare_catalog(gw_ctx *ctx, int64_t n, const double *m1, const double *m2,
                             const double *chi1, const double *chi2, const double *lam1,
                             const double *lam2, const double *dL_Mpc, const uint8_t *zflag,
                             const double *tcoal, const double *fmin,
                             const int32_t *npts_given, int32_t npts_fixed, double per_efold,
                             int32_t npts_lo, int32_t npts_hi,
                             double *Mc, double *eta, double *dL_Gpc, double *chi1o,
                             double *chi2o, double *LamT, double *dLamT, double *tc_s,
                             double *fmax, int32_t *npts, void *stream);

/* Network SNR (Sec. 3.2, Eqs. 3.1-3.2).  DEVICE outputs: snr [n]; snr_det
 * [n_det][n] (per detector; a triangle counts as one detector, its three arms
 * summed in quadrature) or NULL; status [n] or NULL. */
gw_status gw_snr(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                 gw_precision prec, double *snr, double *snr_det, int32_t *status,
                 void *stream);

/* Network Fisher matrix (Sec. 3.2, Eq. 3.3) and SNR.  n_par = 9 (every event
 * pset 0) or 11 (every event pset 1 or 2).  DEVICE outputs:
 *   fisher [n_par(n_par+1)/2][n]: packed upper triangle, row-major over
 *          (i <= j), event-minor (element (i,j) of event e at
 *          fisher[k(i,j) * n + e]), like the paper's (P, P, N) layout;
 *   snr [n] (or NULL); status [n] (or NULL);
 *   grad_params [n_par][n] (or NULL): the SNR vector-Jacobian product of
 *          gw_snr_vjp for the upstream gradient grad_snr [n] (DEVICE), formed
 *          in the same pass.  In the FP64 path it is the exact identity
 *          d SNR/d theta_i = -dL Gamma_{i,dL} / SNR (d h/d dL = -h/dL); the
 *          mixed path accumulates the phase-free sums Re(Q^* dQ/d theta_i). */
gw_status gw_fisher(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                    gw_precision prec, int n_par, double *fisher, double *snr,
                    int32_t *status, const double *grad_snr, double *grad_params,
                    void *stream);

/* Covariance by Cholesky inversion of the normalised Fisher (Sec. 4.1):
 * Gh = Gamma_ij / sqrt(Gamma_ii Gamma_jj), Gh = L L^T, C = Gh^-1 rescaled.
 * Always FP64.  DEVICE in: fisher (layout of gw_fisher), DEVICE out: cov (same
 * layout), cond [n] (1-norm condition number of Gh), inv_err [n]
 * (max_ij |(Gamma C - 1)_ij|), status [n].  Events with cond > cond_max, a
 * non-positive pivot or a non-finite input get NaN outputs. */
gw_status gw_fisher_inverse(gw_ctx *ctx, const double *fisher, int64_t n, int n_par,
                            double cond_max, double *cov, double *cond, double *inv_err,
                            int32_t *status, void *stream);

/* Vector-Jacobian product of the network SNR (derivatives w.r.t. the event's
 * n_par Fisher parameters, same order):
 *   grad_params[i * n + e] = grad_snr[e] * d SNR_e / d theta_i.
 * DEVICE in grad_snr [n]; DEVICE out grad_params [n_par][n]. */
gw_status gw_snr_vjp(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                     gw_precision prec, int n_par, const double *grad_snr,
                     double *grad_params, void *stream);

/* Vector-Jacobian product of L = sum_e log det Gamma_e with respect to the
 * orientation angle gamma_d of every detector d of the network, by Jacobi's
 * formula dL/dgamma = sum_e tr(C_e d Gamma_e/d gamma), with
 * d Gamma/d gamma = 2 Sym(sum W Re(g'^* g^T)) and g' the tangents of the
 * detector rotated by 45 degrees times 2 (the pattern functions are linear in
 * (sin 2 gamma, cos 2 gamma)).  Always FP64 (prec is accepted and ignored): its
 * accuracy is ~1e-16 times the condition number of Gamma.  DEVICE in: cov
 * (layout of gw_fisher_inverse; events whose cov is NaN are skipped);
 * DEVICE out: grad_gamma [n_det] (overwritten).  No counterpart in the paper. */
gw_status gw_logdet_vjp_detangles(gw_ctx *ctx, const gw_catalog *cat,
                                  const gw_network *net, gw_precision prec, int n_par,
                                  const double *cov, double *grad_gamma, void *stream);

/* Allocation-free Fisher pass (no counterpart in the paper).
 *
 * The same computation as gw_fisher (SNR and packed Fisher matrix, same
 * kernels, same results) for callers that cannot allocate device memory while
 * they run: code inside a stream capture that forbids cudaMalloc, applications
 * whose device memory is reserved up front by their own fixed-size pool, or
 * real-time loops that cannot afford an allocation's latency or failure.  It
 * takes no gw_ctx (a context allocates its workspace lazily) and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Workspace: one static device array of GW_NOALLOC_SCRATCH_MIB MiB, held by
 * every GPU that loads the library until the process exits.  It fits about
 * n * (1.6 kB + 0.3 kB per detector) of event constants plus one partial-sum
 * row (~0.6 kB) per work item of at most 256 grid points; a request that does
 * not fit returns GW_ETOOLARGE without computing fisher or snr (status may
 * already hold the per-event checks).  For example, 1e4 events of up to 512
 * points each on one triangle fit.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress,
 * with that device current): make that first call before any stream capture.
 * All calls share the array, so calls that overlap on the GPU (several streams
 * or host threads at once) race and must be serialised by the caller; nothing
 * from an earlier call is read.  Like gw_fisher, it reads back one 8-byte work
 * count (a synchronisation of `stream`).
 * Arguments as gw_fisher; DEVICE outputs fisher [n_par(n_par+1)/2][n] and
 * status [n] are required, snr [n] may be NULL. */
#define GW_NOALLOC_SCRATCH_MIB 32
gw_status gw_fisher_noalloc(const gw_catalog *cat, const gw_network *net, gw_precision prec,
                            int n_par, double *fisher, double *snr, int32_t *status,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GWFISH_H */
