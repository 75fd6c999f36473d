/*
 * cetra.h — C ABI of the GB300 (sm_103a) CETRA transit search library.
 *
 * The library implements the two GPU stages of CETRA (Smith et al. 2025):
 * the linear search (Sec. 2.2: a weighted least-squares template fit at every
 * trial (duration, mid-time) window, Eq. 1 and Eq. 2) and the periodic search
 * (Sec. 2.3: the linear grid phase-folded over trial periods with a common
 * depth, Eq. 3 and Eq. 4, reduced in-kernel to the maximum per period).
 *
 * Conventions for every entry point
 *  - Times and durations are in days (FP64). Flux and flux error are FP32;
 *    flux is normalised to a baseline of 1 unless params.flux_is_offset is
 *    set (then 0 is baseline and positive values are deficits, Sec. 2).
 *  - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *    pointers are CUDA device memory on the context's device, owned by the
 *    caller, and are only touched in stream order on the context's stream.
 *  - Linear-search arrays are [n_dur][n_t0], row-major, t0 contiguous. The
 *    t0 grid is t_i = t_ref + (i p - n_pad q) c / q, i = 0 .. n_t0-1, where c
 *    is the resample cadence, s = c p / q the realised t0 step, and n_pad the
 *    null padding of Sec. 2.1.1 (see cetra_plan_info).
 *  - Null results (a window with no data, Sec. 2.2; a period with no valid
 *    window) are NaN; their indices are -1.
 *  - Every function returns a cetra_status; on failure cetra_last_error(ctx)
 *    gives a one-line message. No entry point aborts the process or leaves
 *    the device in an error state on invalid input.
 *  - A context may be used by one host thread at a time.
 */
#ifndef CETRA_H
#define CETRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CETRA_OK = 0,
    CETRA_EINVAL = 1,    /* invalid argument (sizes, grids, template, no usable points) */
    CETRA_ENOMEM = 2,    /* host or device allocation failed */
    CETRA_ECUDA = 3,     /* a CUDA call or kernel launch failed */
    CETRA_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    CETRA_ECAPACITY = 5  /* an output or workspace buffer is too small */
} cetra_status;

#define CETRA_FP32 0        /* plain FP32 window and fold sums */
#define CETRA_FP32_KAHAN 1  /* Kahan-compensated FP32 sums */

typedef struct cetra_ctx cetra_ctx;
typedef struct cetra_plan cetra_plan;
typedef struct cetra_linear_grid cetra_linear_grid;

/* Search parameters (Sec. 2.1). Zero / negative values select the paper's defaults. */
typedef struct {
    double cadence;        /* resample cadence c (days); <= 0: median input cadence (Sec. 2.1.1) */
    double t0_step;        /* t0 step s (days); <= 0: 1 % of the shortest duration (Sec. 2.1.3).
                              Realised as s = c p / q with 1 <= q <= 64 (smallest q within 1e-9
                              relative, else the closest), so that every index is exact. */
    int template_samples;  /* L, samples of the resampled template (Sec. 2.1.2); <= 0: 1024 */
    int flux_is_offset;    /* 0: flux has baseline 1 and y = 1 - f; 1: flux is already y */
    int precision;         /* CETRA_FP32 or CETRA_FP32_KAHAN */
} cetra_params;

/* Geometry of a plan (Sec. 2.1.1, Sec. 2.1.3). */
typedef struct {
    double t_ref;          /* smallest kept input time (days, absolute) */
    double cadence;        /* c */
    double t0_step;        /* s = c p / q */
    int64_t p, q;          /* s / c = p / q */
    int64_t n_pad;         /* null points padded at each end: ceil((max D / 2) / c) */
    int64_t n_grid;        /* resampled grid length N_g */
    int64_t n_t0;          /* t0 grid length I */
    int64_t n_kept;        /* input points kept (finite t, f, sigma and sigma > 0) */
    int32_t n_dur;         /* J */
    int32_t template_samples;
    int64_t table_entries; /* window-table entries staged by the linear kernel */
    size_t grid_bytes;     /* workspace bytes needed without a periodic search */
} cetra_plan_info;

/* Fill *p with the defaults (median cadence, 1 % t0 step, L = 1024, baseline-1 flux, FP32). */
void cetra_params_default(cetra_params *p);

/*
 * Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
 * the library launches on (NULL: the legacy default stream). The context owns
 * no large buffers until a host-buffer entry point needs them.
 * Errors: CETRA_EINVAL (ctx NULL), CETRA_ECUDA (bad device).
 */
int cetra_create(cetra_ctx **ctx, int device, void *cuda_stream);
/* Release a context. The objects made with it (plans, grids, batches, networks) may be
 * released before or after it, but none may be used once it is gone. */
void cetra_destroy(cetra_ctx *ctx);
/* Change the stream of a context (e.g. to a torch stream). */
int cetra_set_stream(cetra_ctx *ctx, void *cuda_stream);
/* Message of the last failure on this context ("" if none). Owned by ctx. */
const char *cetra_last_error(const cetra_ctx *ctx);
/* Number of kernels this context has launched since creation. */
int64_t cetra_kernel_launches(const cetra_ctx *ctx);

/*
 * Per-kernel timing (a tracing aid, not in the paper). While enabled, every
 * launch is bracketed by a pair of CUDA events on the context's stream.
 * cetra_profile_read synchronises on the recorded events of one kernel
 * ("resample", "linear", "fold", "finalize", "logl0"), returns the number of
 * timed launches and their summed device time in milliseconds, and forgets
 * them. Errors: CETRA_EINVAL (unknown name), CETRA_ECUDA.
 */
int cetra_profile_enable(cetra_ctx *ctx, int enable);
int cetra_profile_read(cetra_ctx *ctx, const char *kernel, int64_t *launches, double *total_ms);

/*
 * Build a plan: the geometry of the resampled light curve and of the t0 grid
 * (Sec. 2.1.1, Sec. 2.1.3) from the host times, and the per-duration window
 * tables of the nearest template sample (Sec. 2.1.2), uploaded to the device.
 *   time/flux/flux_err  host, n_points each; invalid points (non-finite or
 *                       sigma <= 0) are ignored.
 *   durations           host, n_dur > 0 trial durations D_j (days, > 0).
 *   tmpl                host, tmpl_len >= 1 samples of the transit model
 *                       from first to last contact; resampled to L samples by
 *                       linear interpolation and divided by its largest
 *                       absolute value.
 * The plan is owned by the caller (cetra_plan_destroy) and may be reused for
 * any light curve with the same t_ref, cadence and extent.
 * Errors: CETRA_EINVAL (no usable point, cadence undefined, bad durations or
 * template), CETRA_ENOMEM, CETRA_ECUDA.
 */
int cetra_plan_create(cetra_ctx *ctx, const cetra_params *params, const double *time,
                      const float *flux, const float *flux_err, int64_t n_points,
                      const double *durations, int n_dur, const float *tmpl, int tmpl_len,
                      cetra_plan **plan);
int cetra_plan_get_info(const cetra_plan *plan, cetra_plan_info *info);

/*
 * Geometry only (Sec. 2.1.1, Sec. 2.1.3), computed on the host with no device
 * work: what cetra_plan_create would report in cetra_plan_info, without the
 * template tables (table_entries = 0). Lets a caller size the [n_dur][n_t0]
 * outputs of cetra_linear_search before calling it. ctx may be NULL (no
 * message is then recorded). Errors as cetra_plan_create.
 */
int cetra_plan_geometry(cetra_ctx *ctx, const cetra_params *params, const double *time,
                        const float *flux, const float *flux_err, int64_t n_points,
                        const double *durations, int n_dur, cetra_plan_info *info);
void cetra_plan_destroy(cetra_plan *plan);

/* Bytes of device workspace that the device entry points need for n_periods
 * periods (n_periods = 0: the resample and linear stages only). */
size_t cetra_workspace_bytes(const cetra_plan *plan, int n_periods);

/*
 * Device path, stage 1 (Sec. 2.1.1): resample the device light curve onto the
 * plan's grid inside `d_workspace` (nearest grid point; inverse-variance
 * combination; empty points null). d_time (FP64), d_flux, d_flux_err (FP32)
 * are device arrays of n_points. Points that fall outside the plan's grid are
 * dropped. Stream-ordered; returns after the launches are queued.
 * Errors: CETRA_EINVAL (NULL pointers, n_points < 0), CETRA_ECUDA.
 */
int cetra_resample_device(cetra_ctx *ctx, const cetra_plan *plan, const double *d_time,
                          const float *d_flux, const float *d_flux_err, int64_t n_points,
                          void *d_workspace, size_t workspace_bytes);

/*
 * Device path, stage 2 (Sec. 2.2): the linear search over the resampled grid
 * in `d_workspace`. Leaves the per-window sufficient statistics
 * (A = sum m W y, B = sum m^2 W) in the workspace for the periodic stage, and
 * optionally writes the paper's three outputs (Sec. 2.2): depth = A / B,
 * depth_var = 1 / B, dlogl = A^2 / (2 B) (which equals Eq. 2 at the
 * maximum-likelihood depth). d_depth, d_depth_var, d_dlogl: device FP32
 * [n_dur][n_t0] arrays, each may be NULL. Null windows give NaN.
 * Errors: CETRA_EINVAL, CETRA_ECAPACITY (workspace too small), CETRA_ECUDA.
 */
int cetra_linear_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                        size_t workspace_bytes, float *d_depth, float *d_depth_var,
                        float *d_dlogl);

/*
 * Device path, stage 3 (Sec. 2.3): fold the linear grid over the trial
 * periods d_periods (device FP64, n_periods) with the common-depth model and
 * reduce in-kernel to the maximum-likelihood window per period. Only D_j < P_k
 * is evaluated (Sec. 2.3); d_mask (device uint8 [n_periods][n_dur], NULL for
 * none) can exclude further (D, P) pairs. Epoch cells are the nearest t0
 * points t_i + e P (Sec. 2.3). Ties go to the smallest duration index, then
 * the smallest t0 index. Per-period outputs (device arrays of n_periods):
 * d_dlogl, d_t0 (mid-time, absolute days), d_duration, d_depth (common depth
 * Z), d_depth_var (var of Z) as FP64, d_i (t0 index, int64), d_j (duration
 * index, int32). Winners are re-summed in FP64. Any output may be NULL.
 * Errors: CETRA_EINVAL, CETRA_ECAPACITY, CETRA_ECUDA.
 */
int cetra_periodic_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                          size_t workspace_bytes, const double *d_periods, int n_periods,
                          const uint8_t *d_mask, double *d_dlogl, double *d_t0,
                          double *d_duration, double *d_depth, double *d_depth_var,
                          int64_t *d_i, int32_t *d_j);

/*
 * Allocation-free variant of cetra_periodic_device (the paper has no
 * counterpart; this is a deployment aid). For callers that cannot allocate
 * device memory while they run: a fixed memory pool, device buffers handed in
 * by a host application with its own allocator, or a workspace sized once for
 * the linear grid (n_periods = 0) and then reused for period grids of any
 * length. The fold's per-period keys and status word live in a static device
 * array inside the library (CETRA_STATIC_MAX_PERIODS keys + 256 B, about
 * 2 MiB, held by every GPU that loads the library until the process exits)
 * instead of in d_workspace, so d_workspace needs only
 * cetra_workspace_bytes(plan, 0) bytes and must hold a linear grid from
 * cetra_linear_device. Arguments, outputs and tie rules are those of
 * cetra_periodic_device. The call allocates nothing. Every call looks up the
 * array's device address with the context's device current (no allocation);
 * the first call on a device may load the library's device code, so make it
 * before any stream capture. Calls on one device share the array: calls whose
 * kernels overlap on the GPU race and must be serialised by the caller. The
 * status word is cleared at the start of every call; a fold whose bounded
 * device-side wait gave up sets it to CETRA_ETIMEOUT and leaves NaN outputs
 * (and indices -1) for every period. Read it with cetra_static_status.
 * Errors: CETRA_ECAPACITY (n_periods > CETRA_STATIC_MAX_PERIODS, or the
 * workspace is smaller than the linear grid), CETRA_EINVAL, CETRA_ECUDA.
 */
#define CETRA_STATIC_MAX_PERIODS 262144
int cetra_periodic_device_static(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                                 size_t workspace_bytes, const double *d_periods, int n_periods,
                                 const uint8_t *d_mask, double *d_dlogl, double *d_t0,
                                 double *d_duration, double *d_depth, double *d_depth_var,
                                 int64_t *d_i, int32_t *d_j);

/*
 * Status word of the static array after cetra_periodic_device_static on ctx's device: 0, or
 * CETRA_ETIMEOUT if a bounded device-side wait of that call's fold gave up (its outputs are
 * then NaN). Waits for ctx's stream, then copies the word to *status; allocates nothing.
 * The word belongs to the last call on this device from any context.
 * Errors: CETRA_EINVAL (NULL argument), CETRA_ECUDA.
 */
int cetra_static_status(cetra_ctx *ctx, int *status);

/*
 * Self-test of the allocation-free path's failure report (not in the paper): clears the
 * static status word of ctx's device, then queues on ctx's stream one kernel whose bounded
 * barrier wait cannot complete; when the wait gives up (after about a second) the kernel
 * stores CETRA_ETIMEOUT in the static status word, exactly as a fold whose wait gave up
 * does. cetra_static_status then reports it; the next cetra_periodic_device_static clears it.
 * Returns after queueing. Errors: CETRA_EINVAL (NULL ctx), CETRA_ECUDA.
 */
int cetra_selftest_static_timeout(cetra_ctx *ctx);

/*
 * Status word of a workspace after cetra_periodic_device: 0, or CETRA_ETIMEOUT
 * if a bounded device-side wait of the fold gave up (its outputs are then NaN).
 * Synchronises the context's stream.
 */
int cetra_workspace_status(cetra_ctx *ctx, const cetra_plan *plan, const void *d_workspace,
                           size_t workspace_bytes, int *status);

/*
 * Constant-flux log-likelihood (Sec. 2.2, last paragraph): Eq. 1 at zero depth
 * over the non-null grid points of the resampled curve in d_workspace, written
 * to *d_logl0 (device FP64). Adding it to any dlogl gives the whole-curve
 * log-likelihood of that model.
 */
int cetra_logl0_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                       size_t workspace_bytes, double *d_logl0);

/*
 * Host-buffer API: the linear search of Sec. 2.2 on a light curve in host
 * memory. Copies the inputs in, runs resample + linear search, copies the
 * three [n_dur][n_t0] FP32 outputs out (each may be NULL), and returns the
 * device-resident grid in *grid_out (may be NULL) for cetra_periodic_search.
 * *n_t0: in: capacity of each output row set (elements per duration row);
 * out: I. If the capacity is too small nothing is written to the outputs and
 * CETRA_ECAPACITY is returned with *n_t0 = I.
 * The grid owns its device memory until cetra_grid_free.
 */
int cetra_linear_search(cetra_ctx *ctx, const cetra_params *params, const double *time,
                        const float *flux, const float *flux_err, int64_t n_points,
                        const double *durations, int n_dur, const float *tmpl, int tmpl_len,
                        cetra_linear_grid **grid_out, float *depth, float *depth_var,
                        float *dlogl, int64_t *n_t0);

/*
 * Host-buffer API: the periodic search of Sec. 2.3 on a grid returned by
 * cetra_linear_search. periods (host FP64, n_periods), dur_mask (host uint8
 * [n_periods][n_dur] or NULL). Per-period host outputs (each may be NULL):
 * dlogl, t0, duration, depth, depth_var (FP64). *best_k (may be NULL): the
 * period with the largest dlogl (ties: smallest k), -1 if all are null.
 */
int cetra_periodic_search(cetra_ctx *ctx, cetra_linear_grid *grid, const double *periods,
                          int n_periods, const uint8_t *dur_mask, double *dlogl, double *t0,
                          double *duration, double *depth, double *depth_var, int64_t *best_k);

/* ---------------------------------------------------------------------------------------
 * Batched form: many light curves of uneven length, each searched with the linear and the
 * periodic search of Sec. 2.2 and Sec. 2.3, in one launch per stage (a persistent fold
 * kernel drains a work queue of (curve, 8-period group) items), replayed as a CUDA graph.
 * Curves share the cadence, the t0 step, the durations and the template; each has its own
 * time span and its own period grid
 *     P_k = period_min * ratio^k,  k = 0, 1, ... while P_k <= period_max,
 * with ratio^k evaluated in FP64 by least-significant-bit-first square-and-multiply
 * (x = 1, b = ratio; for each bit of k: if set x = x * b; b = b * b).
 * ------------------------------------------------------------------------------------- */
typedef struct cetra_batch cetra_batch;

/* Best periodic model of one curve (Sec. 2.3), re-summed in FP64. */
typedef struct {
    double dlogl;      /* LR of the best (period, t0, duration); NaN if the curve has none */
    double period;     /* days */
    double t0;         /* mid-time of a transit, absolute days */
    double duration;   /* days */
    double depth;      /* common depth Z */
    double depth_var;  /* variance of Z */
    int64_t k;         /* index in the curve's period grid, -1 if null */
    int64_t i;         /* t0 index in the curve's own grid, -1 if null */
    int32_t j;         /* duration index, -1 if null */
    int32_t n_periods; /* periods searched for this curve */
} cetra_best;

typedef struct {
    int32_t n_curves;
    int32_t n_dur;
    int64_t n_points;     /* input points (all curves) */
    int64_t n_cells;      /* resampled cells (all curves) */
    int64_t n_t0;         /* t0 points (all curves) */
    int64_t n_periods;    /* periods (all curves) */
    int64_t n_fold_items; /* (curve, 8-period group) work items of the fold */
    int64_t fold_cell_reads; /* algorithmic (A, B) reads of the fold */
    size_t device_bytes;  /* device memory the batch holds */
    int32_t linear_threads;  /* chosen linear block size */
    int32_t fold_variant;    /* chosen fold shape: bit 0 set = 2 phases per thread (else 4),
                                bit 1 set = at most 4 periods folded together (else 8) */
    int32_t fold_blocks;     /* persistent fold blocks */
    int32_t graph;           /* 1 once the run is captured as a CUDA graph */
    double cadence;          /* shared resample cadence c (days) */
    double t0_step;          /* shared realised t0 step s = c p / q (days) */
    int64_t p, q, n_pad;     /* shared t0 ticks and null padding (see cetra_plan_info) */
} cetra_batch_info;

/*
 * Build a batch: copy the curves to the device, lay out every curve's grids, and (autotune
 * != 0) time the candidate tile shapes of the linear and fold kernels on this batch and keep
 * the fastest. offsets: host int64 [n_curves + 1], curve c owns points
 * [offsets[c], offsets[c+1]) of time (FP64), flux and flux_err (FP32). params->cadence and
 * params->t0_step must be > 0 (shared by all curves). period_min: host [n_curves], > 0.
 * period_max: host [n_curves] or NULL (half the curve's time span); ratio: host [n_curves]
 * or NULL (1 + min(durations) / (2 x time span)), each > 1. The batch owns its device memory
 * (cetra_batch_destroy). Errors: CETRA_EINVAL, CETRA_ENOMEM, CETRA_ECUDA.
 */
int cetra_batch_create(cetra_ctx *ctx, const cetra_params *params, int n_curves,
                       const int64_t *offsets, const double *time, const float *flux,
                       const float *flux_err, const double *durations, int n_dur,
                       const float *tmpl, int tmpl_len, const double *period_min,
                       const double *period_max, const double *period_ratio, int autotune,
                       cetra_batch **batch);
/* Run the whole search of every curve (captured as a CUDA graph on the first call, replayed
 * after) and copy the per-curve results to `best` (host [n_curves], may be NULL). Blocks
 * until done. Errors: CETRA_ECUDA, CETRA_ETIMEOUT (a bounded device wait ran out). */
int cetra_batch_run(cetra_ctx *ctx, cetra_batch *batch, cetra_best *best);
int cetra_batch_get_info(const cetra_batch *batch, cetra_batch_info *info);
void cetra_batch_destroy(cetra_batch *batch);

/*
 * Linear-search features of every curve (resample + linear search, Sec. 2.2): the window
 * likelihood ratio A^2/(2B) of the windows with a positive depth (A > 0), max-pooled over
 * n_bins equal bins of each curve's t0 grid (bin width ceil(n_t0 / n_bins)); empty bins,
 * null windows and negative depths give 0. d_features: device FP32
 * [n_curves][n_dur][n_bins], caller-owned. Blocks until done. (Input of the learned
 * period-interval proposal, which is not in the paper.)
 */
int cetra_batch_features(cetra_ctx *ctx, cetra_batch *batch, int n_bins, float *d_features);

/*
 * Fold only the listed work items and report each curve's best over them. An item is one
 * group of 8 consecutive periods of one curve: curve c's items are
 * first_item(c) .. first_item(c) + ceil(n_periods(c) / 8) - 1 (cetra_batch_curve), item x
 * covering periods 8 (x - first_item(c)) .. + 7. items: host int64 [n_items]. linear != 0
 * reruns the resample and linear stages first (needed unless cetra_batch_features or a
 * run has just left this batch's grids). best as in cetra_batch_run (a curve none of whose
 * items is listed is null). Blocks until done.
 */
int cetra_batch_run_items(cetra_ctx *ctx, cetra_batch *batch, const int64_t *items,
                          int64_t n_items, int linear, cetra_best *best);

/* Geometry and period grid of curve `curve` of a batch (outputs may be NULL). */
int cetra_batch_curve(const cetra_batch *batch, int curve, double *t_ref, double *period_min,
                      double *period_ratio, int32_t *n_periods, int32_t *n_t0,
                      int64_t *first_item);

/*
 * Fold the periods a proposal chose (learned period-interval proposal; not in the paper) and
 * report each curve's best over them. d_scores: device FP32 [n_curves][n_intervals]
 * (cetra_cnn_comb's output), interval q spanning [e_q, e_{q+1}) days with
 * e_q = p_lo (p_hi/p_lo)^(q/n_intervals). Per curve, on the device: of the intervals holding
 * at least one of its periods (n_present), the max(1, ceil(top_frac n_present)) with the
 * highest scores are kept (NaN ranks lowest; ties: lower interval first); every 8-period
 * group holding a period of a kept interval is folded (periods outside [p_lo, p_hi) are never
 * chosen). linear != 0 reruns the resample and linear stages first. Outputs (host, each may be
 * NULL): best [n_curves]; *n_items_out = groups folded; *n_periods_out = periods in them;
 * items_out (capacity n_fold_items) = the folded work items, in no fixed order. Blocks until
 * done. Errors: CETRA_EINVAL (n_intervals outside 1..1024, p_lo <= 0, p_hi <= p_lo,
 * top_frac outside (0, 1]), CETRA_ECUDA, CETRA_ETIMEOUT.
 */
int cetra_batch_run_proposed(cetra_ctx *ctx, cetra_batch *batch, const float *d_scores,
                             int n_intervals, double p_lo, double p_hi, double top_frac,
                             int linear, cetra_best *best, int64_t *n_items_out,
                             int64_t *n_periods_out, int64_t *items_out);

/* One-shot batched search: cetra_batch_create (no autotuning) + cetra_batch_run +
 * cetra_batch_destroy. */
int cetra_search_batch(cetra_ctx *ctx, const cetra_params *params, int n_curves,
                       const int64_t *offsets, const double *time, const float *flux,
                       const float *flux_err, const double *durations, int n_dur,
                       const float *tmpl, int tmpl_len, const double *period_min,
                       const double *period_max, const double *period_ratio, cetra_best *best);

/* ---------------------------------------------------------------------------------------
 * Learned period-interval proposal (not in the paper): a 1-D CNN over a curve's max-pooled
 * linear-search likelihood ratios [n_dur][n_bins] (cetra_batch_features) that marks the bins
 * holding transits, and a comb that turns that map into scores of log-spaced period
 * intervals, so that the fold can evaluate the most promising intervals only. Network:
 * log1p(x) -> conv(in -> 32, k 9) ReLU -> conv(32 -> 32) ReLU -> conv(32 -> 32) ReLU ->
 * conv(32 -> 1), zero padding; FP32 training copy of the weights, BF16 weights in every
 * kernel, FP32 sums. Parameters (flat FP32): for each layer W [out][in][9] then b [out].
 * ------------------------------------------------------------------------------------- */
typedef struct cetra_cnn cetra_cnn;

/* Create a network for in_channels 1..32 (the durations) and n_bins (a multiple of 256) per
 * curve, He-normal initial weights from `seed` (zero biases); the network owns device buffers
 * for max_batch curves (activations, gradients, Adam state). Blocks. Errors: CETRA_EINVAL
 * (sizes), CETRA_ENOMEM, CETRA_ECUDA. Release with cetra_cnn_destroy (NULL allowed). */
int cetra_cnn_create(cetra_ctx *ctx, int in_channels, int n_bins, int max_batch, uint64_t seed,
                     cetra_cnn **cnn);
void cetra_cnn_destroy(cetra_cnn *cnn);
/* Number of FP32 parameters (the length of host_params / host_grads below). */
int64_t cetra_cnn_param_count(const cetra_cnn *cnn);
/* The sizes a network was created with (each output may be NULL). */
int cetra_cnn_shape(const cetra_cnn *cnn, int *in_channels, int *n_bins, int *max_batch);
/* Copy the FP32 training copy of the parameters to host_params (caller-owned). Blocks. */
int cetra_cnn_get_params(cetra_ctx *ctx, const cetra_cnn *cnn, float *host_params);
/* Replace the parameters from host_params, re-round the BF16 weights and reset the optimiser
 * state (moments and step count). Blocks. */
int cetra_cnn_set_params(cetra_ctx *ctx, cetra_cnn *cnn, const float *host_params);
/* Probabilities for B <= max_batch curves: d_features device FP32 [B][in][n_bins] (read only),
 * d_prob device FP32 [B][n_bins] (written), both caller-owned. Asynchronous on the context's
 * stream. Errors: CETRA_EINVAL (NULL pointers, B outside 1..max_batch), CETRA_ECUDA. */
int cetra_cnn_forward(cetra_ctx *ctx, cetra_cnn *cnn, const float *d_features, int B,
                      float *d_prob);
/* Forward + backward of the weighted binary cross-entropy with logits against d_labels
 * (device FP32 [B][n_bins], 0 or 1), mean over bins, positive weight pos_weight. Leaves the
 * gradient on the device for cetra_cnn_adam; *loss and host_grads (flat, like the
 * parameters) are filled when not NULL (that synchronises). Weight gradients are summed with
 * atomics, so their last bits may differ from run to run. Errors as cetra_cnn_forward. */
int cetra_cnn_backward(cetra_ctx *ctx, cetra_cnn *cnn, const float *d_features,
                       const float *d_labels, int B, float pos_weight, double *loss,
                       float *host_grads);
/* One bias-corrected Adam step with the last gradient on the FP32 parameters, then the BF16
 * weights are re-rounded. Asynchronous. */
int cetra_cnn_adam(cetra_ctx *ctx, cetra_cnn *cnn, float lr, float beta1, float beta2,
                   float eps);
/* Proposal map d_map[b][t] = d_prob[b][t] * max_j max(d_features[b][j][t], 0): the network's
 * transit probability times the bin's best window likelihood ratio (Sec. 2.2). d_prob, d_map: device FP32 [B][n_bins]; d_features: device FP32
 * [B][n_dur][n_bins] (cetra_batch_features). Asynchronous on the context's stream. */
int cetra_cnn_map(cetra_ctx *ctx, const float *d_prob, const float *d_features, int B,
                  int n_dur, int n_bins, float *d_map);
/* Comb scores of n_intervals log-spaced period intervals between p_lo and p_hi days for each
 * of B per-bin maps d_map [B][n_bins]. Curve b has V_b = d_n_valid[b] valid bins (device
 * int32 [B]; NULL means n_bins) of d_bin_days[b] days (device FP64 [B]). Interval q spans
 * p_lo (p_hi/p_lo)^(q/n) .. p_lo (p_hi/p_lo)^((q+1)/n); in bins [blo, bhi), its trials are the
 * midpoints of max(1, ceil((bhi - blo) V_b / blo)) equal parts (the last epoch's phase moves
 * by about one bin between neighbouring trials), skipped below 1 bin or above V_b / 2. For a
 * trial P (F = floor(P 2^32 + 1/2)) and a phase ph < ceil(P), the epochs are
 * t_e = (ph 2^32 + e F + 2^31) >> 32 < V_b and the score is sum_e map[t_e] / sqrt(E); the
 * interval's score is the best of those, 0 if none is positive or if the bin width is <= 0.
 * d_scores: device FP32 [B][n_intervals]. Asynchronous on the context's stream.
 * Errors: CETRA_EINVAL (NULL pointers, B outside 1..65535, n_bins outside 1..2^30,
 * n_intervals < 1, p_lo <= 0, p_hi <= p_lo). */
int cetra_cnn_comb(cetra_ctx *ctx, const float *d_map, int B, int n_bins,
                   const double *d_bin_days, const int *d_n_valid, double p_lo, double p_hi,
                   int n_intervals, float *d_scores);

/* The whole learned-proposal search of a batch in one call (not in the paper): resample and
 * linear stages, features (cetra_batch_features at the network's n_bins), the network's
 * probabilities (in chunks of its max_batch), the map, the comb over n_intervals intervals
 * between p_lo and p_hi (p_hi <= 0: just above the batch's longest trial period), and
 * cetra_batch_run_proposed with top_frac. The network must have n_dur input channels. Device
 * scratch (features, maps, scores: about n_curves x (n_dur + 2) x n_bins x 4 bytes) is allocated
 * and freed by the call. Outputs as cetra_batch_run_proposed. Blocks.
 * Errors: CETRA_EINVAL (arguments, channel mismatch), CETRA_ENOMEM, CETRA_ECUDA, CETRA_ETIMEOUT. */
int cetra_batch_search_proposed(cetra_ctx *ctx, cetra_batch *batch, cetra_cnn *cnn,
                                int n_intervals, double p_lo, double p_hi, double top_frac,
                                cetra_best *best, int64_t *n_items_out, int64_t *n_periods_out);


/* ---------------------------------------------------------------------------------------
 * Method neighbours of the search.
 *
 * Masking (Sec. 4.2: before each further search of a curve, the flux in and around the best
 * signal of the previous search is nulled). The mask acts on the resampled grid: cell k, at
 * time g_k = t_ref + (k - n_pad) c, is nulled (W y = W = 0) when |g_k - (t0 + n P)| < h for
 * its nearest epoch n = floor((g_k - t0) / P + 1/2), evaluated in FP64 with one rounding per
 * operation. h is half the masked width (days).
 *
 * Single-transit (monotransit) events (Sec. 1 and Sec. 5: single transits are searched for
 * in the linear-search output): greedily, the window (i, j) with the largest LR among the
 * windows with a positive depth whose t0 index is not hidden by an earlier event e, hidden
 * meaning |i - i_e| < D_{j_e} q / (c p) (FP64: the event's duration in t0 steps); ties go to
 * the smallest j, then the smallest i.
 * ------------------------------------------------------------------------------------- */
#define CETRA_MAX_EVENTS 4096

typedef struct {
    double dlogl;      /* the window's LR, A^2 / (2B), from its FP32 sums in FP64 */
    double t0;         /* mid-time, absolute days */
    double duration;   /* days */
    double depth;      /* A / B */
    double depth_var;  /* 1 / B */
    int64_t i;         /* t0 index */
    int32_t j;         /* duration index */
    int32_t pad_;
} cetra_event;

/* Device path: null the cells of the resampled grid in `d_workspace` (from
 * cetra_resample_device) within half_width days of the mid-times t0 + n period. Rerun
 * cetra_linear_device afterwards. d_n_masked (device, may be NULL) is increased by the number
 * of nulled cells that held data. half_width = 0 does nothing. Asynchronous.
 * Errors: CETRA_EINVAL (period <= 0 or not finite, t0 not finite, half_width < 0),
 * CETRA_ECAPACITY (workspace smaller than cetra_workspace_bytes(plan, 0)). */
int cetra_mask_transits_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                               size_t workspace_bytes, double period, double t0,
                               double half_width, unsigned long long *d_n_masked);

/* Host path: mask a grid from cetra_linear_search (as above) and rerun its linear stage, so
 * that the next cetra_periodic_search / cetra_monotransit_search sees the masked curve.
 * *n_masked (may be NULL) = nulled cells that held data. Blocks until done. */
int cetra_mask_transits(cetra_ctx *ctx, cetra_linear_grid *grid, double period, double t0,
                        double half_width, int64_t *n_masked);

/* Bytes of workspace cetra_monotransits_device needs (>= cetra_workspace_bytes(plan, 0)). */
size_t cetra_monotransit_workspace_bytes(const cetra_plan *plan, int max_events);

/* Device path: up to max_events single-transit events (strongest first) from the linear grid
 * in d_workspace (cetra_linear_device), into d_events (device, max_events) and *d_n_events
 * (device int). Asynchronous. Errors: CETRA_EINVAL (max_events outside 1..4096),
 * CETRA_ECAPACITY (workspace below cetra_monotransit_workspace_bytes; n_t0 > 2^24 or more
 * than 256 durations). */
int cetra_monotransits_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                              size_t workspace_bytes, int max_events, cetra_event *d_events,
                              int *d_n_events);

/* Host path: the same on a grid from cetra_linear_search; events (host, max_events) and
 * *n_events filled. Blocks until done. */
int cetra_monotransit_search(cetra_ctx *ctx, cetra_linear_grid *grid, int max_events,
                             cetra_event *events, int *n_events);

/* Iterative search (Sec. 4.2): n_iter rounds of cetra_periodic_search on the grid, each round
 * after the first on the curve with the previous round's best signal masked over
 * width x its duration (width <= 0: 2, i.e. within one duration of each mid-time). out
 * (host, n_iter) gets each round's best model (k its period index, j its duration index,
 * i = -1); *n_found = rounds that found a model. The grid is left masked. Blocks. */
int cetra_search_iterative(cetra_ctx *ctx, cetra_linear_grid *grid, const double *periods,
                           int n_periods, const uint8_t *dur_mask, int n_iter, double width,
                           cetra_best *out, int *n_found);

/* Self-test of the bounded waits (the fold's barrier waits give up after about 2e9 SM clocks,
 * record CETRA_ETIMEOUT and return instead of hanging): one kernel waits on a barrier that
 * expects bytes no copy delivers. *timed_out = 1 when the wait gave up as designed, *seconds =
 * the kernel's duration (may be NULL). Blocks for about a second; the context stays usable. */
int cetra_selftest_wait_timeout(cetra_ctx *ctx, int *timed_out, double *seconds);

/* Measured ceilings for the roofline denominators of the two stages: the window sums of the
 * linear search (Sec. 2.2) are packed FP32 FMAs, and the fold (Sec. 2.3) is one 8-byte
 * shared-memory load plus one packed FP32 add per cell read. Runs two microbenchmark kernels
 * on ctx's stream, one full wave of blocks each, timed with CUDA events after a warm-up launch
 * (best of three):
 *   *fma_tflops  independent fma.rn.f32x2 chains, 2 flop per FMA lane, in TFLOP/s;
 *   *smem_gbs    conflict-free 8-byte shared-memory loads, each added into a packed FP32 sum,
 *                in GB/s of bytes loaded.
 * Either pointer may be NULL. Blocks for some tens of ms. Returns CETRA_OK, CETRA_EINVAL (NULL
 * ctx), CETRA_ENOMEM or CETRA_ECUDA. */
int cetra_measure_peaks(cetra_ctx *ctx, double *fma_tflops, double *smem_gbs);

/* Release a grid from cetra_linear_search (NULL is allowed). */
void cetra_grid_free(cetra_linear_grid *grid);

/* Geometry of a grid from cetra_linear_search. */
int cetra_grid_get_info(const cetra_linear_grid *grid, cetra_plan_info *info);

#ifdef __cplusplus
}
#endif

#endif /* CETRA_H */
