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
    GW_MIXED = 1,  /* FP64 grid, phase derivatives, tau*, Earth angle and
                      accumulation; FP32 amplitude, patterns, tangents and
                      products with exactly compensated (double-float) sums  */
    GW_DFLOAT = 2  /* Fisher pass of networks with at most two interferometers
                      per grid point (one triangle, or up to two L-shaped
                      detectors): every per-point quantity in double-float
                      arithmetic (pairs of FP32, ~2^-48) on the FP32 pipe, the
                      Gram matrix of the tangents (rounded to 49 bits relative
                      to their column's largest value, seven digits) exact on
                      the tensor cores (see gw_set_fp64_gram), rounded once to
                      FP64; results of the FP64 accuracy class.  Every other pass and wider networks
                      run as GW_FP64.  Not accepted by gw_set_tile,
                      gw_autotune or gw_fisher_noalloc. */
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
    GW_ST_OVERFLOW = 64,    /* work items beyond the gw_reserve capacity       */
    GW_ST_SVD_FALLBACK = 128 /* gw_covariance: not positive definite, inverted
                               by the SVD instead (GW_INV_CHO_SVD)             */
};

/* A work item is a run of at most GW_ITEM_POINTS consecutive grid points of one
 * event: an event of npts points has ceil(npts / GW_ITEM_POINTS) items.  The
 * Fisher pass with its Gram on the tensor cores (GW_DFLOAT, or GW_FP64 after
 * gw_set_fp64_gram(ctx, 1), on networks of at most two interferometers per
 * grid point) takes items of GW_TC_ITEM_POINTS points: ceil(npts / 128). */
#define GW_ITEM_POINTS 256
#define GW_TC_ITEM_POINTS 128

/* Fisher parameter order (the fixed order of Sec. 3.2): slot 0..8 =
 *   Mc [Msun, detector frame], eta, dL [Gpc], theta, phi, iota, psi [rad],
 *   tc [s], Phic [rad];
 * slots 9, 10 depend on the event's parameter set:
 *   pset 1 -> chi1z, chi2z;  pset 2 -> LambdaTilde, deltaLambdaTilde.
 * pset 0 events have 9 parameters. */

/* Catalog: structure of arrays, every pointer DEVICE, read only.  The call
 * processes n events; event i of the call is row r(i) of the columns, with
 * r(i) = sel[i] when sel is given (the columns then hold at least
 * max(sel) + 1 rows; sel need not be sorted) and r(i) = i otherwise.  Every
 * per-event output is indexed by i.
 *
 * Duty factor (Sec. 3.2, and the duty_factor option of Sec. 5): each detector,
 * and each arm of a triangle separately, is on or off for a whole event.
 * arm_mask[r] bit a = 1 when arm a of the network is on for row r, the arms
 * being numbered over the detectors in order (an L-shaped detector one arm, a
 * triangle three, k = 0, 1, 2); NULL = every arm on.  The random draws are the
 * caller's.  An event with every arm off has SNR 0 and a zero Fisher matrix
 * (status 0; the inverse flags it GW_ST_NOT_PD). */
typedef struct gw_catalog {
    int64_t n;
    const double *Mc, *eta, *dL, *theta, *phi, *iota, *psi, *tc, *Phic;
    const double *chi1z, *chi2z;      /* NULL -> 0 (spins enter the phase)    */
    const double *LamT, *dLamT;       /* NULL -> 0 (tidal phase)              */
    const int8_t *pset;               /* 0, 1 or 2 (see above)                */
    const double *fmin, *fmax;        /* grid ends [Hz]                       */
    const int32_t *npts;              /* grid points, log spaced (Sec. 2.2)   */
    const uint32_t *arm_mask;         /* duty-factor arm masks, or NULL       */
    const int64_t *sel;               /* [n] rows to process, or NULL         */
} gw_catalog;

/* Interferometer.  shape 0: L-shaped with opening angle zeta and bisector at
 * gamma counter-clockwise from local East; shape 1: triangle of three
 * co-located 60-degree interferometers (zeta ignored) whose bisectors are at
 * gamma + 30 deg + 120 deg k (Table 2: gamma of a triangle is its first arm).
 * Angles in radians.  psd indexes the network's PSD table.  A network has at
 * most 32 arms and at most 24 interferometer entries (one per L, five per
 * triangle: its two-interferometer form and its three arms). */
typedef struct gw_detector {
    double lat, lon, gamma, zeta;
    int32_t shape, psd;
} gw_detector;

/* Noise PSD of an interferometer (Sec. 3.1: each detector carries its noise
 * curve, given by a file of frequencies and PSD or ASD values, the psd_path
 * and is_ASD options).  Two kinds:
 *  GW_PSD_POWER_SUM: S_n(f) = scale * sum_{j<nterm} coef[j] (f/f0)^pw[j],
 *      1 <= nterm <= 4, coef >= 0, integer powers |pw| <= 15;
 *  GW_PSD_TABLE: S_n(f) = scale * T(f), T the straight line through
 *      (ln f_j, ln T_j) and (ln f_j+1, ln T_j+1) for f_j <= f <= f_j+1 (log-log
 *      linear interpolation of the tabulated curve); T_j = table_s[j], or
 *      table_s[j]^2 when is_asd (the table holds the amplitude spectral
 *      density).  Outside [table_f[0], table_f[n_table-1]] the interferometer
 *      is blind (zero noise weight).  table_f, table_s: DEVICE [n_table],
 *      2 <= n_table <= 2^20, table_f strictly increasing and > 0, table_s > 0,
 *      read during the call (the library builds its log table in the call's
 *      workspace); a table that breaks these rules gives NaN noise weights, so
 *      the events' outputs are NaN.  f0, nterm, coef and pw are ignored. */
enum { GW_PSD_POWER_SUM = 0, GW_PSD_TABLE = 1 };
typedef struct gw_psd {
    double f0, scale;
    int32_t nterm, kind;
    double coef[4], pw[4];
    const double *table_f, *table_s;
    int32_t n_table, is_asd;
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
/* ABI version of this header (incremented on any signature change or addition): 7. */
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

/* Tiles of the Fisher pass (no counterpart in the paper).  The fused point
 * kernels process work items of GW_ITEM_POINTS points with a group of `group`
 * lanes each (4, 8 or 16; default 8) on a persistent grid of `blocks_per_sm`
 * CTAs per SM (1 or 2; default 2).  The context keeps one tile per precision
 * and grid-length class: class 0 = at most ~1.5 work items per event on
 * average (grids up to ~380 points), 1 = up to 12 (~3000 points), 2 = longer;
 * a call's class is its mean work items per event (after gw_reserve: the
 * reservation's max_items / max_events).  Results do not depend on the tile
 * (the reductions keep a fixed order per tile; different tiles sum in
 * different orders, within rounding).
 * gw_set_tile installs a tile; gw_autotune times every tile (group x
 * blocks_per_sm, `reps` Fisher passes each after one warm-up, CUDA events
 * around the point kernel) on the caller's catalog, installs the fastest for
 * the catalog's class and precision, and returns the class, the tile and the
 * six times in ms (ms_out [6]: group 4, 8, 16 x blocks 1, 2; or NULL).  It
 * synchronises `stream` and must not run in the asynchronous mode of
 * gw_reserve. */
gw_status gw_set_tile(gw_ctx *ctx, gw_precision prec, int length_class, int group,
                      int blocks_per_sm);
gw_status gw_autotune(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                      gw_precision prec, int n_par, int reps, int32_t *length_class,
                      int32_t *group, int32_t *blocks_per_sm, double *ms_out, void *stream);

/* Gram accumulation of the FP64 Fisher pass (no counterpart in the paper).
 * tensor = 1: for networks of at most two interferometers per
 * grid point (one triangle, or up to two L-shaped detectors) the pass forms
 * each work item's Gram matrix of tangents (Sec. 3.2, Eq. 3.3) on the tensor
 * cores: every tangent is rounded to a 56-bit fixed-point number relative to
 * the largest exponent of its column in the item, split into eight 7-bit
 * digits, and the digit products are summed exactly (integers below 2^24 in
 * the FP32 accumulator, then the 64 digit-pair sums as 128-bit integers) and
 * rounded once to FP64.  The result is the FP64 Fisher matrix up to that
 * rounding.
 * tensor = 0 (the default): every product on the FP64 pipe, as for wider
 * networks and the other passes (measured slightly faster: without the Gram the
 * FP64 pass is a chain of dependent FP64 operations per point).  GW_DFLOAT
 * always forms its Gram on the tensor cores; the mixed path is not affected. */
gw_status gw_set_fp64_gram(gw_ctx *ctx, int tensor);

/* Kernel fault flag (no counterpart in the paper): the tensor-core kernel
 * bounds every wait on its own MMAs (about a second); a wait that runs out
 * writes NaN into the affected work item's sums, ends that CTA after freeing
 * its tensor memory, and sets this context's flag.  gw_kernel_faults copies the
 * flag (0 or 1) to *faults (HOST) and clears it when `reset` is nonzero;
 * synchronous (waits for the device). */
gw_status gw_kernel_faults(gw_ctx *ctx, int32_t *faults, int reset);

/* Measurement hook (no counterpart in the paper): when enabled, the context
 * records CUDA events on the call's stream around every point-loop kernel
 * launch (the fused SNR / Fisher / VJP kernel).  gw_point_kernel_ms waits for
 * the last recorded pair and returns its duration in milliseconds (negative
 * when nothing was recorded). */
gw_status gw_set_profiling(gw_ctx *ctx, int enable);
double gw_point_kernel_ms(gw_ctx *ctx);

/* Measurement hook (no counterpart in the paper): FMA throughput of the FP64
 * (fp64 = 1) or FP32 (fp64 = 0) pipe of the current device, measured with
 * independent FMA chains in every thread of a grid that fills every SM (each
 * thread runs 8 chains of `iters` FMAs, FP32 as packed FP32x2 FMAs, so 16 FMAs
 * per iteration; 1 <= iters <= 2^24; the launch is repeated once to warm the
 * clocks).  HOST outputs: *fma_per_clk_sm (FMAs per
 * SM clock and SM, from the SM cycle counter), *fma_per_s (FMAs per second
 * over the whole GPU, from CUDA events), *sm_mhz (the SM clock during the
 * loop).  Allocates and frees two small device buffers; synchronises `stream`. */
gw_status gw_fma_rate(int fp64, int iters, double *fma_per_clk_sm, double *fma_per_s,
                      double *sm_mhz, void *stream);

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

/* Detection gate (Sec. 5, the snr_th option: Fisher matrices are computed only
 * for events whose network SNR exceeds the threshold).  DEVICE in: snr [n];
 * DEVICE out: sel [n capacity], the indices i with snr[i] > threshold in
 * increasing order (NaN never passes); HOST out: *n_sel.  Synchronises
 * `stream` to read the count.  The selected events are processed by passing
 * sel (and n = *n_sel) in a gw_catalog. */
gw_status gw_select_snr(gw_ctx *ctx, const double *snr, int64_t n, double threshold,
                        int64_t *sel, int64_t *n_sel, void *stream);

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

/* Precision refinement of a mixed-precision pass (the conditioning check of
 * Sec. 4.1 applied to the precision of the Fisher matrix).  The mixed path's
 * Fisher matrix carries an elementwise error of ~1e-7 of sqrt(Gamma_ii
 * Gamma_jj) (FP32 patterns, amplitudes and tangents), which Gamma^-1 amplifies
 * by up to the condition number; the FP64 path's error is ~1e-14.  After
 * gw_fisher(GW_MIXED) and gw_fisher_inverse on the same events, every event i
 * with status[i] == 0 whose inversion failed (inv_status NOT_PD or NONFINITE)
 * or whose condition number cond[i] exceeds cond_th (or is NaN) is recomputed
 * by the FP64 path (Fisher pass with the fused SNR VJP when grad_snr is given,
 * then the Cholesky inversion with cond_max) and its entries of fisher, snr,
 * status, grad_params, cov, cond, inv_err and inv_status are overwritten; the
 * other events are left untouched.  The refined events' results equal those of
 * gw_fisher(GW_FP64) + gw_fisher_inverse bit for bit.
 * DEVICE in/out (layouts of gw_fisher and gw_fisher_inverse, n = cat->n):
 * fisher, status, cov, cond, inv_status (required); snr, inv_err (or NULL);
 * grad_snr [n] and grad_params [n_par][n] (both or neither).  DEVICE out:
 * refined [n] (or NULL), 1 for the recomputed events.  HOST out: *n_refined
 * (or NULL).  Reads back the number of selected events (a synchronisation of
 * `stream`).  A cond_th of 1e7 keeps the mixed events' sqrt(diag C) within
 * 1e-3 of FP64 on the synthetic catalogs.  No counterpart in the paper. */
gw_status gw_fisher_refine(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, int n_par,
                           double cond_th, double cond_max, double *fisher, double *snr,
                           int32_t *status, const double *grad_snr, double *grad_params,
                           double *cov, double *cond, double *inv_err, int32_t *inv_status,
                           uint8_t *refined, int64_t *n_refined, void *stream);

/* Fisher pass and inversion with the precision chosen per event (no
 * counterpart in the paper; the passes compute Sec. 3.2, Eqs. 3.1-3.3, and the
 * inversion of Sec. 4.1).  Events whose parameter set p has bit p of
 * dfloat_psets set run the double-float pass (GW_DFLOAT); the others run the
 * mixed pass (GW_MIXED) first, then gw_fisher_refine's check: those with a
 * clean point-loop status and a failed inversion or a condition number above
 * cond_th join the double-float events in one double-float pass (FP64
 * accuracy class; FP64 for networks it does not take), whose results are
 * written over their mixed ones.  Every event is inverted with cond_max.  The precision is a per-event property: an
 * event's results equal those of the pass it was routed to (plus, for the
 * mixed events, the double-float recomputation), in the call's event order.  Use it where one
 * class of events is known to be ill-conditioned (here the BBH, whose two spins
 * are nearly degenerate: dfloat_psets = 1 << 1) and the rest is not; the
 * refinement guards the mixed events either way.
 * DEVICE out (layouts of gw_fisher and gw_fisher_inverse, n = cat->n):
 * fisher, status, cov, cond, inv_status (required); snr, inv_err (or NULL);
 * grad_params [n_par][n] with DEVICE in grad_snr [n] (both or neither: the
 * fused SNR VJP).  HOST out: *n_dfloat, the events routed to the double-float
 * pass, and *n_refined, the mixed events recomputed (either may be
 * NULL).  Reads back the split and the double-float pass's event count
 * (synchronisations of `stream`).  Errors as gw_fisher; GW_EINVAL for a NaN cond_th or missing
 * required outputs. */
gw_status gw_fisher_routed(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, int n_par,
                           uint32_t dfloat_psets, double cond_th, double cond_max, double *fisher,
                           double *snr, int32_t *status, const double *grad_snr,
                           double *grad_params, double *cov, double *cond, double *inv_err,
                           int32_t *inv_status, int64_t *n_dfloat, int64_t *n_refined,
                           void *stream);

/* Vector-Jacobian product of the network SNR (Sec. 3.2, Eqs. 3.1-3.2)
 * w.r.t. the event's n_par Fisher parameters (same order):
 *   grad_params[i * n + e] = grad_snr[e] * d SNR_e / d theta_i,
 * and, when grad_gamma is not NULL, w.r.t. the orientation angle gamma_d of
 * every detector d of the network, summed over the events:
 *   grad_gamma[d] = sum_e grad_snr[e] * d SNR_e / d gamma_d
 * (dQ/dgamma follows from the pattern functions being linear in
 * (sin 2 gamma, cos 2 gamma); a triangle's three arms turn together; events
 * with a non-zero status are left out of the sum).
 * DEVICE in grad_snr [n]; DEVICE out grad_params [n_par][n] and grad_gamma
 * [n_det] (or NULL; overwritten).  No counterpart in the paper. */
gw_status gw_snr_vjp(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net,
                     gw_precision prec, int n_par, const double *grad_snr,
                     double *grad_params, double *grad_gamma, void *stream);

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

/* gw_logdet_vjp_detangles for the detectors of det_mask only (bit d: detector d
 * of the network, d < n_det), e.g. the L-shaped detectors of a network whose
 * orientations are being optimised.  A detector's gradient sums only its own
 * interferometers, so the point loop skips the sites of the other detectors
 * (the cost scales with the selected ones) and the selected entries equal
 * those of gw_logdet_vjp_detangles bit for bit.  DEVICE out: grad_gamma [n_det]
 * (overwritten; entries of detectors outside det_mask are NaN).  det_mask with
 * no bit below n_det fails with GW_EINVAL.  No counterpart in the paper. */
gw_status gw_logdet_vjp_detangles_masked(gw_ctx *ctx, const gw_catalog *cat,
                                         const gw_network *net, gw_precision prec, int n_par,
                                         const double *cov, uint32_t det_mask,
                                         double *grad_gamma, void *stream);

/* Detector strain h_a(f_k) = Q_a exp(i Phi_a) on every event's grid, for every
 * arm a of the network (the arm numbering of gw_catalog.arm_mask: a triangle
 * gives its three 60-degree arms), with the conventions of the Fisher pass:
 * Phi = Psi_PN(f) + Psi_tidal(f) - Phic - pi/4 + Phi_D(f) at the fiducial tc
 * (Secs. 2.2 and 3.1).  Phi is evaluated in FP64 and reduced modulo 2 pi by the
 * Cody-Waite method; the sine and cosine of the reduced angle are FP64
 * (GW_FP64) or FP32 (GW_MIXED).  total_points must equal the sum of the
 * events' npts (checked: one read-back, the call synchronises `stream`).
 * DEVICE out: re, im [n_arm][total_points], event e's points at
 * [point_off[e], point_off[e+1]); freq [total_points] (or NULL);
 * point_off [n + 1] (or NULL); status [n] (or NULL).  Arms that are off for
 * the event (duty factor) get zeros; flagged events NaN. */
gw_status gw_strain(gw_ctx *ctx, const gw_catalog *cat, const gw_network *net, gw_precision prec,
                    int64_t total_points, double *re, double *im, double *freq,
                    int64_t *point_off, int32_t *status, void *stream);

/* ---- Covariance tools (Sec. 4.1 and Sec. 4.2).  Matrices are packed like
 * gw_fisher's output ([P(P+1)/2][n], DEVICE); one thread per event, FP64.
 * A keep mask selects parameters: bit i set = slot i kept (0 = all kept); the
 * kept slots, in increasing order, form the output's parameter list. */

/* Inversion methods of gw_covariance (the options of CovMatr, Sec. 4.1). */
typedef enum {
    GW_INV_CHO = 0,        /* Cholesky; not positive definite: GW_ST_NOT_PD, NaN  */
    GW_INV_CHO_SVD = 1,    /* Cholesky, SVD when not positive definite (the
                              paper's default; sets GW_ST_SVD_FALLBACK)          */
    GW_INV_SVD = 2,        /* eigendecomposition (the SVD of a symmetric matrix)  */
    GW_INV_SVD_TRUNC = 3,  /* singular values below thresh * s_max raised to it  */
    GW_INV_SVD_REG = 4,    /* singular values below thresh * s_max left out       */
    GW_INV_LU = 5          /* LU with partial pivoting: the upper triangle of the
                              LU inverse, inv_err of the full LU inverse          */
} gw_inv_method;

/* Eigenvalues (ascending) and eigenvectors of each Fisher matrix, normalised
 * by sqrt(diag) when `normalize` and every diagonal element is positive
 * (CheckFisher, Sec. 4.1).  DEVICE out: eigval [n_par][n] (or NULL), eigvec
 * [n_par * n_par][n] (or NULL): component i of eigenvector k of event e at
 * eigvec[(i * n_par + k) * n + e], largest-magnitude component positive.
 * n_par <= 11.  Cyclic Jacobi in FP64. */
gw_status gw_fisher_eig(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, int normalize,
                        double *eigval, double *eigvec, void *stream);

/* Covariance with the Fisher manipulations of Sec. 4.2 and the inversion
 * options of Sec. 4.1, per event: (1) fixParams: keep the parameters of
 * `keep` (rows and columns of fixed parameters removed before inversion);
 * (2) addPrior: add prior[i] (HOST [n_par] or NULL; finite, >= 0) to the
 * diagonal entry of every kept slot i; (3) normalise by sqrt(diag) unless a
 * diagonal element is not positive; (4) condition number = max|w| / min|w|
 * over the eigenvalues w of the normalised matrix, above cond_max nothing is
 * inverted (GW_ST_COND_GT_MAX, NaN); (5) invert by `method` (thresh in
 * [0, 1): the singular-value floor ratio of methods 3 and 4, the paper's
 * default 1e-15); (6) undo the normalisation; inv_err = max|Gamma C - 1| with
 * the kept, prior-added Gamma.  DEVICE out: cov [Pk(Pk+1)/2][n] over the Pk
 * kept parameters; cond, inv_err, status [n] (each may be NULL). */
gw_status gw_covariance(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, uint32_t keep,
                        const double *prior, int method, double thresh, double cond_max,
                        double *cov, double *cond, double *inv_err, int32_t *status,
                        void *stream);

/* The kept rows and columns of packed matrices: fixing parameters when
 * applied to Fisher matrices, marginalising over the others when applied to
 * covariances (Sec. 4.2).  DEVICE in [n_par(n_par+1)/2][n], DEVICE out
 * [Pk(Pk+1)/2][n]. */
gw_status gw_packed_submatrix(gw_ctx *ctx, const double *in, int64_t n, int n_par, uint32_t keep,
                              double *out, void *stream);

/* perturb_Fisher (Sec. 4.1): every element of the packed Fisher matrices
 * perturbed at the eps-th relative decimal, out = fisher * (1 + eps r), with r
 * the caller's random numbers (DEVICE, same packed layout, e.g. uniform in
 * [-1, 1]: the packed triangle keeps the matrices symmetric).  Inverting out
 * and fisher with gw_covariance and comparing shows whether the inversion is
 * stable.  DEVICE in: fisher, r [n_par(n_par+1)/2][n]; DEVICE out: out (may
 * equal fisher). */
gw_status gw_perturb_fisher(gw_ctx *ctx, const double *fisher, int64_t n, int n_par, double eps,
                            const double *r, double *out, void *stream);

/* Sky-localisation area at confidence level perc (percent, in (0, 100)),
 * Sec. 4.1: Delta Omega = -2 pi |sin theta| sqrt(C_tt C_pp - C_tp^2)
 * ln(1 - perc/100), from the packed covariances (DEVICE [n_par(n_par+1)/2][n])
 * with theta at slot i_theta and phi at slot i_phi; theta DEVICE [n] (rad).
 * units 0: steradians, 1: square degrees.  DEVICE out: area [n]. */
gw_status gw_sky_area(gw_ctx *ctx, const double *cov, int64_t n, int n_par, int i_theta,
                      int i_phi, const double *theta, double perc, int units, double *area,
                      void *stream);

/* Allocation-free Fisher pass (no counterpart in the paper).
 *
 * The same computation as gw_fisher (SNR and packed Fisher matrix, same
 * kernels, same results) for callers that must not allocate device memory
 * while they run: applications that hand all device memory to their own
 * fixed-size pool at start-up (a cudaMalloc would fail or steal from the
 * pool), and long-running or latency-bound loops that cannot afford an
 * allocation's latency, its implicit synchronisation or its possible failure
 * in the middle of a job.  It takes no gw_ctx (a context allocates its
 * workspace lazily) and calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Workspace: one static device array of GW_NOALLOC_SCRATCH_MIB MiB, held by
 * every GPU that loads the library until the process exits.  It fits about
 * n * (1.6 kB + 0.3 kB per detector) of event constants plus one partial-sum
 * row (~0.6 kB) per work item of at most 256 grid points; a request that does
 * not fit returns GW_ETOOLARGE without writing fisher or snr (status may
 * already hold the per-event checks).  For example, 1e4 events of up to 512
 * points each on one triangle fit.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress, with that device current):
 * make that first call before any stream capture on the device.  All calls
 * share the array and each call overwrites what it uses, so calls that overlap
 * on the GPU (several streams or host threads at once) race and must be
 * serialised by the caller; nothing from an earlier call is read.  Like
 * gw_fisher, it reads back one 8-byte work count (a synchronisation of
 * `stream`).
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
