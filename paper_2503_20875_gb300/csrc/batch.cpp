// Batched form of the CETRA search (declarations in include/cetra.h): many light curves of
// uneven length searched together, one launch per stage, replayed as a CUDA graph.
//
// Layout: the curves' input points, resampled cells, (A, B) grids and periods are packed
// back to back (CSR offsets per curve). All curves share the cadence, the t0 step, the
// durations and the template, hence one set of window tables (a plan built from the first
// curve). Each curve has its own time span (t_ref, grid length, t0 count) and period grid.
//
// Work order of the fold: the curves by decreasing t0 count (the largest first), each curve's
// 8-period groups from its longest periods down, so that the queue ends with its cheapest
// items; a curve's items stay together, so the blocks running at the same time read few
// curves' grids (the L2 holds them).
//
// Autotuning (optional, at creation): the linear stage is timed with 128- and 64-thread
// blocks (t0 outputs per block), and the fold in its four shapes (4 or 2 phases per thread,
// sub-groups of at most 8 or 4 periods per block) on a sample of work items spread over the
// whole queue; the fastest of each is kept. The chosen sequence of memsets and kernels is
// captured once into a CUDA graph on the batch's own stream and replayed by every run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

struct cetra_batch {
    cetra_ctx *ctx = nullptr;    // used while the batch runs, never by its destruction
    int device = 0;
    cetra_plan *plan = nullptr;  // shared geometry constants and window tables
    int n_curves = 0;
    std::vector<batch_curve> curves;
    std::vector<int64_t> pt_off, tile_off, group_off;
    int64_t n_points = 0, n_cells = 0, n_t0 = 0, n_periods = 0, n_tiles = 0, n_items = 0;
    int64_t ab_cells = 0, fold_cell_reads = 0;
    int lin_threads = 128, fold_variant = 0, fold_blocks = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    // device memory
    void *d_mem = nullptr;
    size_t d_bytes = 0;
    double *d_time = nullptr;
    float *d_flux = nullptr, *d_err = nullptr;
    float2 *d_grid = nullptr;  // interleaved (W y, W) cells of every curve
    float2 *d_ab = nullptr;
    int64_t *d_pt_off = nullptr, *d_tile_off = nullptr, *d_group_off = nullptr;
    batch_curve *d_curves = nullptr;
    unsigned long long *d_keys = nullptr, *d_pkeys = nullptr;
    cetra_best *d_best = nullptr;
    int *d_queue = nullptr, *d_status = nullptr;
    int64_t *d_items = nullptr;  // explicit fold work list (cetra_batch_run_items)
    int64_t *d_order_off = nullptr;   // queue order: items before each curve of the order
    int32_t *d_order_curve = nullptr;  // queue order: the curves, largest first
    unsigned char *d_flags = nullptr;        // one byte per work item (proposal selection)
    unsigned long long *d_counts = nullptr;  // selected items, their periods
};

namespace {

bool usable(double t, float f, float e) {
    return std::isfinite(t) && std::isfinite(f) && std::isfinite(e) && e > 0.0f;
}

// Number of k >= 0 with batch_period_host(pmin, ratio, k) <= pmax (the grid grows with k).
int64_t period_count(double pmin, double ratio, double pmax) {
    if (!(pmin > 0.0) || !(ratio > 1.0) || !(pmax >= pmin) || !std::isfinite(pmax)) return 0;
    double est = std::floor(std::log(pmax / pmin) / std::log(ratio)) + 1.0;
    int64_t K = est > 0 ? (int64_t)est : 1;
    while (batch_period_host(pmin, ratio, K) <= pmax) ++K;
    while (K > 0 && batch_period_host(pmin, ratio, K - 1) > pmax) --K;
    return K;
}

int fail(cetra_ctx *ctx, int code, const char *msg) { return set_error(ctx, code, msg); }

int cuda_fail(cetra_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, CETRA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Tile list of the linear stage for `threads`-wide blocks.
int64_t build_tiles(cetra_batch *b, int threads) {
    const int64_t UT = (int64_t)threads * LIN_RB, q = b->plan->q;
    b->tile_off.assign((size_t)b->n_curves + 1, 0);
    for (int c = 0; c < b->n_curves; ++c) {
        const int64_t I = b->curves[c].I;
        const int64_t U = (I + q - 1) / q;
        b->tile_off[c + 1] = b->tile_off[c] + (I > 0 ? (U + UT - 1) / UT : 0);
    }
    return b->tile_off.back();
}

// Algorithmic (A, B) reads of the fold of one curve: about I reads per (period, duration
// D < P) (each t0 cell belongs to one (phase, epoch) of a period, up to the rounding of
// the epoch offsets at the ends), over the periods of at least one t0 step. The periods
// ascend, so per duration the periods above it are a suffix of the grid: O(J) per curve.
int64_t fold_reads(const cetra_plan *plan, const batch_curve &cv) {
    const int64_t K = cv.n_periods;
    if (K <= 0 || cv.I <= 0) return 0;
    const double s = plan->cadence * (double)plan->p / (double)plan->q;  // t0 step, days
    const int64_t below_step = period_count(cv.pmin, cv.ratio, std::nextafter(s, 0.0));
    int64_t total = 0;
    for (double D : plan->durations) {
        const int64_t upto = std::max(period_count(cv.pmin, cv.ratio, D), below_step);
        total += (int64_t)cv.I * std::max<int64_t>(0, K - std::min(K, upto));
    }
    return total;
}

// The stages before the fold: clear, resample, linear search.
cudaError_t enqueue_linear(cetra_batch *b, int lin_threads) {
    cetra_plan *plan = b->plan;
    cudaStream_t st = b->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->d_grid, 0, (size_t)b->n_cells * sizeof(float2), st))) return e;
    if ((e = cudaMemsetAsync(b->d_status + 1, 0, sizeof(int), st))) return e;  // linear status
    if ((e = cudaMemsetAsync(b->d_ab, 0, (size_t)b->ab_cells * sizeof(float2), st))) return e;
    if ((e = launch_batch_resample(st, b->ctx->num_sms, plan, b->d_time, b->d_flux, b->d_err,
                                   b->n_points, b->d_pt_off, b->n_curves, b->d_curves,
                                   b->d_grid)))
        return e;
    return launch_batch_linear(st, plan, lin_threads, b->d_tile_off, b->n_curves, b->n_tiles,
                               b->d_curves, b->d_grid, b->d_ab, b->d_status + 1);
}

// The fold over n_items work items (item_list NULL: items 0 .. n_items-1; n_items_dev not
// NULL: the first *n_items_dev entries of item_list, at most n_items) and the finalize.
cudaError_t enqueue_fold(cetra_batch *b, int64_t n_items, int fold_variant,
                         const int64_t *item_list,
                         const unsigned long long *n_items_dev = nullptr) {
    cetra_plan *plan = b->plan;
    cudaStream_t st = b->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->d_keys, 0, (size_t)b->n_curves * sizeof(unsigned long long), st)))
        return e;
    if ((e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), st))) return e;  // queue, status
    if ((e = launch_batch_fold(st, b->fold_blocks, fold_variant, plan, b->d_ab, b->d_curves,
                               b->d_group_off, b->n_curves, n_items, b->d_queue, b->d_pkeys,
                               b->d_keys, b->d_status, item_list, n_items_dev, b->d_order_off,
                               b->d_order_curve)))
        return e;
    return launch_batch_finalize(st, plan, b->d_ab, b->d_curves, b->n_curves, b->d_pkeys,
                                 b->d_keys, b->d_status, b->d_best);
}

cudaError_t enqueue(cetra_batch *b, int64_t n_items, int fold_variant, int lin_threads,
                    const int64_t *item_list = nullptr) {
    cudaError_t e = enqueue_linear(b, lin_threads);
    if (e) return e;
    return enqueue_fold(b, n_items, fold_variant, item_list);
}

// Milliseconds of one enqueue() with the given shapes (the batch is rebuilt by the caller);
// item_list: the fold's work items (NULL: the queue order).
int time_once(cetra_batch *b, int64_t n_items, int fold_variant, int lin_threads, float *ms,
              const int64_t *item_list = nullptr) {
    cudaError_t e = cudaEventRecord(b->ev_start, b->stream);
    if (!e) e = enqueue(b, n_items, fold_variant, lin_threads, item_list);
    if (!e) e = cudaEventRecord(b->ev_stop, b->stream);
    if (!e) e = cudaEventSynchronize(b->ev_stop);
    if (!e) e = cudaEventElapsedTime(ms, b->ev_start, b->ev_stop);
    if (e) return cuda_fail(b->ctx, e, "batch autotune");
    return CETRA_OK;
}

int upload_tiles(cetra_batch *b) {
    cudaError_t e = cudaMemcpy(b->d_tile_off, b->tile_off.data(),
                               b->tile_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    return e ? cuda_fail(b->ctx, e, "batch tiles") : CETRA_OK;
}

int autotune(cetra_batch *b) {
    // linear block size: time the whole run without the fold (n_items = 0)
    float best_ms = 0.f;
    int best_threads = 128;
    for (int threads : {128, 64}) {
        b->n_tiles = build_tiles(b, threads);
        int rc = upload_tiles(b);
        if (rc) return rc;
        float ms = 0.f;
        if ((rc = time_once(b, 0, 0, threads, &ms))) return rc;  // warm-up
        if ((rc = time_once(b, 0, 0, threads, &ms))) return rc;
        if (threads == 128 || ms < best_ms) {
            best_ms = ms;
            best_threads = threads;
        }
    }
    b->lin_threads = best_threads;
    b->n_tiles = build_tiles(b, best_threads);
    int rc = upload_tiles(b);
    if (rc) return rc;
    if (b->plan->precision == CETRA_FP32_KAHAN) return CETRA_OK;  // one fold shape
    // fold shape: time a sample of work items spread evenly over the whole batch (every
    // stride-th item: all curve lengths, all period ranges) with each variant
    const int64_t sample = std::min<int64_t>(b->n_items, (int64_t)b->fold_blocks * 8);
    if (sample <= 0) return CETRA_OK;
    std::vector<int64_t> picks((size_t)sample);
    for (int64_t x = 0; x < sample; ++x) picks[(size_t)x] = x * b->n_items / sample;
    cudaError_t ce = cudaMemcpy(b->d_items, picks.data(), (size_t)sample * sizeof(int64_t),
                                cudaMemcpyHostToDevice);
    if (ce) return cuda_fail(b->ctx, ce, "batch autotune sample");
    float base = 0.f;
    if ((rc = time_once(b, 0, 0, best_threads, &base))) return rc;
    float best_fold = 0.f;
    for (int v = 0; v < batch_fold_variants(); ++v) {
        float ms = 0.f;
        if ((rc = time_once(b, sample, v, best_threads, &ms, b->d_items))) return rc;
        if ((rc = time_once(b, sample, v, best_threads, &ms, b->d_items))) return rc;
        ms -= base;
        if (v == 0 || ms < best_fold) {
            best_fold = ms;
            b->fold_variant = v;
        }
    }
    return CETRA_OK;
}

void release(cetra_batch *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_stop) cudaEventDestroy(b->ev_stop);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaFree(b->d_mem);
    if (b->plan) cetra_plan_destroy(b->plan);
    delete b;
}

}  // namespace

extern "C" {

int cetra_batch_create(cetra_ctx *ctx, const cetra_params *params, int n_curves,
                       const int64_t *offsets, const double *time, const float *flux,
                       const float *flux_err, const double *durations, int n_dur,
                       const float *tmpl, int tmpl_len, const double *period_min,
                       const double *period_max, const double *period_ratio, int autotune_on,
                       cetra_batch **out) {
    if (!ctx || !out) return set_error(ctx, CETRA_EINVAL, "batch: NULL ctx or batch");
    *out = nullptr;
    if (!params || !offsets || !time || !flux || !flux_err || !durations || !tmpl || !period_min)
        return fail(ctx, CETRA_EINVAL, "batch: NULL input pointer");
    if (n_curves < 1) return fail(ctx, CETRA_EINVAL, "batch: n_curves < 1");
    if (!(params->cadence > 0.0) || !(params->t0_step > 0.0))
        return fail(ctx, CETRA_EINVAL, "batch: params.cadence and params.t0_step must be > 0");
    const int64_t n_points = offsets[n_curves] - offsets[0];
    if (offsets[0] != 0 || n_points < 0) return fail(ctx, CETRA_EINVAL, "batch: bad offsets");
    for (int c = 0; c < n_curves; ++c)
        if (offsets[c + 1] < offsets[c]) return fail(ctx, CETRA_EINVAL, "batch: offsets decrease");

    cetra_batch *b = new (std::nothrow) cetra_batch;
    if (!b) return fail(ctx, CETRA_ENOMEM, "batch: host allocation");
    b->ctx = ctx;
    b->device = ctx->device;
    b->n_curves = n_curves;
    b->n_points = n_points;
    auto bail = [&](int rc) {
        release(b);
        return rc;
    };

    // shared plan (window tables, n_pad, p/q) from the first curve that has two usable points
    int64_t first = -1;
    for (int c = 0; c < n_curves && first < 0; ++c) {
        int good = 0;
        for (int64_t k = offsets[c]; k < offsets[c + 1] && good < 2; ++k)
            good += usable(time[k], flux[k], flux_err[k]);
        if (good >= 1) first = c;
    }
    if (first < 0) return bail(fail(ctx, CETRA_EINVAL, "batch: no curve has a usable point"));
    int rc = cetra_plan_create(ctx, params, time + offsets[first], flux + offsets[first],
                               flux_err + offsets[first], offsets[first + 1] - offsets[first],
                               durations, n_dur, tmpl, tmpl_len, &b->plan);
    if (rc) return bail(rc);
    cetra_plan *plan = b->plan;
    const double c = plan->cadence;
    const double dmin = *std::min_element(durations, durations + n_dur);

    // per-curve geometry (Sec. 2.1.1, Sec. 2.1.3) and period grid
    b->curves.resize(n_curves);
    b->pt_off.assign(offsets, offsets + n_curves + 1);
    b->group_off.assign((size_t)n_curves + 1, 0);
    int64_t grid = 0, abc = 0, t0s = 0, per = 0;
    for (int cidx = 0; cidx < n_curves; ++cidx) {
        batch_curve cv{};
        cv.pt_off = offsets[cidx];
        double t_ref = INFINITY, t_max = -INFINITY;
        for (int64_t k = offsets[cidx]; k < offsets[cidx + 1]; ++k)
            if (usable(time[k], flux[k], flux_err[k])) {
                t_ref = std::min(t_ref, time[k]);
                t_max = std::max(t_max, time[k]);
            }
        if (std::isfinite(t_ref)) {
            const double tau_max = t_max - t_ref;
            const int64_t ng = 2 * plan->n_pad + (int64_t)std::floor(tau_max / c + 0.5) + 1;
            const int64_t I = ((ng - 1) * plan->q) / plan->p + 1;
            if (ng > INT32_MAX / 2 || I > INT32_MAX / 2 || I * (int64_t)n_dur > (int64_t)UINT32_MAX)
                return bail(fail(ctx, CETRA_EINVAL, "batch: a curve's grid is too large"));
            cv.t_ref = t_ref;
            cv.n_grid = (int32_t)ng;
            cv.I = (int32_t)I;
            cv.ld = ((I + FOLD_PAD) + 1) & ~(int64_t)1;
            const double pmin = period_min[cidx];
            const double pmax = period_max ? period_max[cidx] : 0.5 * tau_max;
            const double ratio = period_ratio ? period_ratio[cidx]
                                              : 1.0 + dmin / (2.0 * std::max(tau_max, dmin));
            if (!(pmin > 0.0) || !(ratio > 1.0) || !std::isfinite(ratio))
                return bail(fail(ctx, CETRA_EINVAL, "batch: period_min must be > 0 and ratio > 1"));
            const int64_t K = period_count(pmin, ratio, pmax);
            if (K > (int64_t)INT32_MAX / 2)
                return bail(fail(ctx, CETRA_EINVAL, "batch: too many periods in one curve"));
            cv.pmin = pmin;
            cv.ratio = ratio;
            cv.n_periods = (int32_t)K;
        }
        cv.grid_off = grid;
        cv.ab_off = abc;
        cv.per_off = per;
        grid += (cv.n_grid + 1) & ~1;  // each curve's cells start on a 16-byte boundary
        abc += (int64_t)n_dur * cv.ld;
        t0s += cv.I;
        per += cv.n_periods;
        b->group_off[cidx + 1] = b->group_off[cidx] + (cv.n_periods + FT_G - 1) / FT_G;
        b->curves[cidx] = cv;
    }
    b->n_cells = grid;
    b->ab_cells = abc;
    b->n_t0 = t0s;
    b->n_periods = per;
    b->n_items = b->group_off.back();
    for (const auto &cv : b->curves) b->fold_cell_reads += fold_reads(plan, cv);

    // device memory, one allocation carved in 256-byte aligned pieces
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0, o_time, o_flux, o_err, o_grid, o_ab, o_pt, o_tile, o_grp, o_cv, o_keys,
                    o_pkeys, o_best, o_q, o_items, o_flags, o_cnt;
    o_time = off; off = up(off + (size_t)n_points * sizeof(double));
    o_flux = off; off = up(off + (size_t)n_points * sizeof(float));
    o_err = off; off = up(off + (size_t)n_points * sizeof(float));
    o_grid = off; off = up(off + (size_t)grid * sizeof(float2));
    o_ab = off; off = up(off + (size_t)abc * sizeof(float2));
    o_pt = off; off = up(off + (size_t)(n_curves + 1) * sizeof(int64_t));
    o_tile = off; off = up(off + (size_t)(n_curves + 1) * sizeof(int64_t));
    o_grp = off; off = up(off + (size_t)(n_curves + 1) * sizeof(int64_t));
    o_cv = off; off = up(off + (size_t)n_curves * sizeof(batch_curve));
    o_keys = off; off = up(off + (size_t)n_curves * sizeof(unsigned long long));
    o_pkeys = off; off = up(off + (size_t)std::max<int64_t>(per, 1) * sizeof(unsigned long long));
    o_best = off; off = up(off + (size_t)n_curves * sizeof(cetra_best));
    o_q = off; off = up(off + 3 * sizeof(int));  // queue, fold status, linear status
    o_items = off; off = up(off + (size_t)std::max<int64_t>(b->n_items, 1) * sizeof(int64_t));
    o_flags = off; off = up(off + (size_t)std::max<int64_t>(b->n_items, 1));
    o_cnt = off; off = up(off + 2 * sizeof(unsigned long long));
    const size_t o_ooff = off;
    off = up(off + (size_t)(n_curves + 1) * sizeof(int64_t));
    const size_t o_ocur = off;
    off = up(off + (size_t)n_curves * sizeof(int32_t));
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (e) return bail(cuda_fail(ctx, e, "batch device"));
    e = cudaMalloc(&b->d_mem, off);
    if (e) {
        b->d_mem = nullptr;
        return bail(fail(ctx, CETRA_ENOMEM, "batch: device allocation"));
    }
    b->d_bytes = off;
    char *base = static_cast<char *>(b->d_mem);
    b->d_time = reinterpret_cast<double *>(base + o_time);
    b->d_flux = reinterpret_cast<float *>(base + o_flux);
    b->d_err = reinterpret_cast<float *>(base + o_err);
    b->d_grid = reinterpret_cast<float2 *>(base + o_grid);
    b->d_ab = reinterpret_cast<float2 *>(base + o_ab);
    b->d_pt_off = reinterpret_cast<int64_t *>(base + o_pt);
    b->d_tile_off = reinterpret_cast<int64_t *>(base + o_tile);
    b->d_group_off = reinterpret_cast<int64_t *>(base + o_grp);
    b->d_curves = reinterpret_cast<batch_curve *>(base + o_cv);
    b->d_keys = reinterpret_cast<unsigned long long *>(base + o_keys);
    b->d_pkeys = reinterpret_cast<unsigned long long *>(base + o_pkeys);
    b->d_best = reinterpret_cast<cetra_best *>(base + o_best);
    b->d_queue = reinterpret_cast<int *>(base + o_q);
    b->d_status = b->d_queue + 1;
    b->d_items = reinterpret_cast<int64_t *>(base + o_items);
    b->d_flags = reinterpret_cast<unsigned char *>(base + o_flags);
    b->d_counts = reinterpret_cast<unsigned long long *>(base + o_cnt);
    b->d_order_off = reinterpret_cast<int64_t *>(base + o_ooff);
    b->d_order_curve = reinterpret_cast<int32_t *>(base + o_ocur);
    // queue order: curves by decreasing t0 count (ties: curve index)
    std::vector<int32_t> order((size_t)n_curves);
    for (int cidx = 0; cidx < n_curves; ++cidx) order[(size_t)cidx] = cidx;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return b->curves[(size_t)x].I > b->curves[(size_t)y].I;
    });
    std::vector<int64_t> order_off((size_t)n_curves + 1, 0);
    for (int k = 0; k < n_curves; ++k) {
        const int32_t cidx = order[(size_t)k];
        order_off[(size_t)k + 1] =
            order_off[(size_t)k] + (b->group_off[(size_t)cidx + 1] - b->group_off[(size_t)cidx]);
    }

    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) ||
        (e = cudaEventCreate(&b->ev_start)) || (e = cudaEventCreate(&b->ev_stop)))
        return bail(cuda_fail(ctx, e, "batch stream"));
    const size_t nb = (size_t)n_points;
    if ((e = cudaMemcpy(b->d_time, time, nb * sizeof(double), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_flux, flux, nb * sizeof(float), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_err, flux_err, nb * sizeof(float), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_pt_off, b->pt_off.data(), b->pt_off.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_group_off, b->group_off.data(), b->group_off.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_curves, b->curves.data(), b->curves.size() * sizeof(batch_curve),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_order_off, order_off.data(), order_off.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_order_curve, order.data(), order.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)))
        return bail(cuda_fail(ctx, e, "batch upload"));
    if ((e = batch_configure(plan))) return bail(cuda_fail(ctx, e, "batch configure"));
    b->fold_blocks = ctx->num_sms * FT_MIN_BLOCKS;
    b->lin_threads = 128;
    b->n_tiles = build_tiles(b, 128);
    if ((rc = upload_tiles(b))) return bail(rc);
    if (autotune_on && (rc = autotune(b))) return bail(rc);
    *out = b;
    return CETRA_OK;
}

int cetra_batch_run(cetra_ctx *ctx, cetra_batch *b, cetra_best *best) {
    if (!ctx || !b) return set_error(ctx, CETRA_EINVAL, "batch_run: NULL argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (e) return cuda_fail(ctx, e, "batch_run device");
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            cudaError_t le = enqueue(b, b->n_items, b->fold_variant, b->lin_threads);
            e = cudaStreamEndCapture(b->stream, &g);
            if (!e) e = le;
        }
        if (!e) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e) {
            b->graph = nullptr;
            return cuda_fail(ctx, e, "batch graph capture");
        }
    }
    // order after the caller's stream, run, and let the caller's stream wait for the batch
    if ((e = cudaEventRecord(b->ev_start, ctx->stream)) ||
        (e = cudaStreamWaitEvent(b->stream, b->ev_start, 0)) ||
        (e = cudaGraphLaunch(b->graph, b->stream)))
        return cuda_fail(ctx, e, "batch graph launch");
    ctx->launches += 4;
    int status[2] = {0, 0};  // fold, linear stage
    if (best && (e = cudaMemcpyAsync(best, b->d_best, (size_t)b->n_curves * sizeof(cetra_best),
                                     cudaMemcpyDeviceToHost, b->stream)))
        return cuda_fail(ctx, e, "batch results");
    if ((e = cudaMemcpyAsync(status, b->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream)) ||
        (e = cudaStreamSynchronize(b->stream)))
        return cuda_fail(ctx, e, "batch run");
    if (status[0] || status[1]) return set_error(ctx, CETRA_ETIMEOUT, "batch_run: a device wait timed out");
    return CETRA_OK;
}

int cetra_batch_features(cetra_ctx *ctx, cetra_batch *b, int n_bins, float *d_features) {
    if (!ctx || !b || !d_features || n_bins < 1)
        return set_error(ctx, CETRA_EINVAL, "batch_features: bad argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaEventRecord(b->ev_start, ctx->stream);
    if (!e) e = cudaStreamWaitEvent(b->stream, b->ev_start, 0);
    if (!e) e = enqueue_linear(b, b->lin_threads);
    if (!e) e = launch_batch_features(b->stream, ctx->num_sms, b->plan, b->d_ab, b->d_curves,
                                      b->n_curves, n_bins, d_features);
    if (!e) e = cudaStreamSynchronize(b->stream);
    if (e) return cuda_fail(ctx, e, "batch_features");
    ctx->launches += 3;
    return CETRA_OK;
}

int cetra_batch_run_items(cetra_ctx *ctx, cetra_batch *b, const int64_t *items, int64_t n_items,
                          int linear, cetra_best *best) {
    if (!ctx || !b || n_items < 0 || (n_items > 0 && !items))
        return set_error(ctx, CETRA_EINVAL, "batch_run_items: bad argument");
    if (n_items > b->n_items)
        return set_error(ctx, CETRA_ECAPACITY, "batch_run_items: more items than the batch has");
    for (int64_t x = 0; x < n_items; ++x)
        if (items[x] < 0 || items[x] >= b->n_items)
            return set_error(ctx, CETRA_EINVAL, "batch_run_items: item out of range");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaEventRecord(b->ev_start, ctx->stream);
    if (!e) e = cudaStreamWaitEvent(b->stream, b->ev_start, 0);
    if (!e && n_items)
        e = cudaMemcpyAsync(b->d_items, items, (size_t)n_items * sizeof(int64_t),
                            cudaMemcpyHostToDevice, b->stream);
    if (!e && linear) e = enqueue_linear(b, b->lin_threads);
    if (!e) e = enqueue_fold(b, n_items, b->fold_variant, b->d_items);
    int status[2] = {0, 0};  // fold, linear stage
    if (!e && best)
        e = cudaMemcpyAsync(best, b->d_best, (size_t)b->n_curves * sizeof(cetra_best),
                            cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaMemcpyAsync(status, b->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaStreamSynchronize(b->stream);
    if (e) return cuda_fail(ctx, e, "batch_run_items");
    ctx->launches += linear ? 4 : 2;
    if (status[0] || status[1]) return set_error(ctx, CETRA_ETIMEOUT, "batch_run_items: a device wait timed out");
    return CETRA_OK;
}

int cetra_batch_run_proposed(cetra_ctx *ctx, cetra_batch *b, const float *d_scores,
                             int n_intervals, double p_lo, double p_hi, double top_frac,
                             int linear, cetra_best *best, int64_t *n_items_out,
                             int64_t *n_periods_out, int64_t *items_out) {
    if (!ctx || !b || !d_scores || n_intervals < 1 || n_intervals > SEL_MAX_INTERVALS ||
        !(p_lo > 0.0) || !(p_hi > p_lo) || !std::isfinite(p_hi) || !(top_frac > 0.0) ||
        !(top_frac <= 1.0))
        return set_error(ctx, CETRA_EINVAL, "batch_run_proposed: bad argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaEventRecord(b->ev_start, ctx->stream);
    if (!e) e = cudaStreamWaitEvent(b->stream, b->ev_start, 0);
    if (!e && linear) e = enqueue_linear(b, b->lin_threads);
    if (!e) e = cudaMemsetAsync(b->d_counts, 0, 2 * sizeof(unsigned long long), b->stream);
    if (!e)
        e = launch_batch_select(b->stream, b->d_curves, b->d_group_off, b->n_curves, d_scores,
                                n_intervals, p_lo, p_hi, top_frac, b->d_flags, b->d_items,
                                b->d_counts);
    if (!e) e = enqueue_fold(b, b->n_items, b->fold_variant, b->d_items, b->d_counts);
    unsigned long long counts[2] = {0, 0};
    int status[2] = {0, 0};  // fold, linear stage
    if (!e && best)
        e = cudaMemcpyAsync(best, b->d_best, (size_t)b->n_curves * sizeof(cetra_best),
                            cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaMemcpyAsync(counts, b->d_counts, sizeof(counts), cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaMemcpyAsync(status, b->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaStreamSynchronize(b->stream);
    if (!e && items_out && counts[0])
        e = cudaMemcpy(items_out, b->d_items, (size_t)counts[0] * sizeof(int64_t),
                       cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(ctx, e, "batch_run_proposed");
    ctx->launches += linear ? 5 : 3;
    if (n_items_out) *n_items_out = (int64_t)counts[0];
    if (n_periods_out) *n_periods_out = (int64_t)counts[1];
    if (status[0] || status[1])
        return set_error(ctx, CETRA_ETIMEOUT, "batch_run_proposed: a device wait timed out");
    return CETRA_OK;
}

int cetra_batch_search_proposed(cetra_ctx *ctx, cetra_batch *b, cetra_cnn *cnn, int n_intervals,
                                double p_lo, double p_hi, double top_frac, cetra_best *best,
                                int64_t *n_items_out, int64_t *n_periods_out) {
    if (!ctx || !b || !cnn || n_intervals < 1 || n_intervals > SEL_MAX_INTERVALS || !(p_lo > 0.0))
        return set_error(ctx, CETRA_EINVAL, "batch_search_proposed: bad argument");
    int cin = 0, T = 0, mb = 0;
    cetra_cnn_shape(cnn, &cin, &T, &mb);
    const int J = b->plan->J, n = b->n_curves;
    if (cin != J) return set_error(ctx, CETRA_EINVAL, "batch_search_proposed: network channels != durations");
    if (!(p_hi > 0.0)) {  // just above the longest trial period of the batch
        p_hi = 0.0;
        for (const auto &cv : b->curves)
            if (cv.n_periods > 0)
                p_hi = std::max(p_hi, batch_period_host(cv.pmin, cv.ratio, cv.n_periods - 1));
        p_hi = p_hi > 0.0 ? p_hi * (1.0 + 1e-9) : 2.0 * p_lo;
    }
    // per-curve bin width (days) and valid bins of the features
    std::vector<double> bw((size_t)n, 0.0);
    std::vector<int> nv((size_t)n, 0);
    for (int c = 0; c < n; ++c) {
        const int64_t I = b->curves[(size_t)c].I;
        if (I <= 0) continue;
        const int64_t width = (I + T - 1) / T;
        bw[(size_t)c] = (double)width * b->plan->t0_step;
        nv[(size_t)c] = (int)((I + width - 1) / width);
    }
    const size_t nf = (size_t)n * J * T, nm = (size_t)n * T, ns = (size_t)n * n_intervals;
    char *mem = nullptr;
    const size_t bytes = (nf + 2 * nm + ns) * sizeof(float) + (size_t)n * (sizeof(double) + sizeof(int)) + 1024;
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e && cudaMalloc((void **)&mem, bytes) != cudaSuccess)
        return set_error(ctx, CETRA_ENOMEM, "batch_search_proposed: device scratch");
    float *feat = reinterpret_cast<float *>(mem);
    float *prob = feat + nf, *map = prob + nm, *scores = map + nm;
    double *d_bw = reinterpret_cast<double *>(scores + ns);
    int *d_nv = reinterpret_cast<int *>(d_bw + n);
    int rc = CETRA_OK;
    if (!e) e = cudaMemcpyAsync(d_bw, bw.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(d_nv, nv.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    if (e) rc = cuda_fail(ctx, e, "batch_search_proposed");
    if (rc == CETRA_OK) rc = cetra_batch_features(ctx, b, T, feat);
    for (int a = 0; rc == CETRA_OK && a < n; a += mb)
        rc = cetra_cnn_forward(ctx, cnn, feat + (size_t)a * J * T, std::min(mb, n - a),
                               prob + (size_t)a * T);
    if (rc == CETRA_OK) rc = cetra_cnn_map(ctx, prob, feat, n, J, T, map);
    if (rc == CETRA_OK)
        rc = cetra_cnn_comb(ctx, map, n, T, d_bw, d_nv, p_lo, p_hi, n_intervals, scores);
    if (rc == CETRA_OK)
        rc = cetra_batch_run_proposed(ctx, b, scores, n_intervals, p_lo, p_hi, top_frac, 0, best,
                                      n_items_out, n_periods_out, nullptr);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(mem);
    return rc;
}

int cetra_batch_curve(const cetra_batch *b, int curve, double *t_ref, double *period_min,
                      double *period_ratio, int32_t *n_periods, int32_t *n_t0,
                      int64_t *first_item) {
    if (!b || curve < 0 || curve >= b->n_curves) return CETRA_EINVAL;
    const batch_curve &cv = b->curves[curve];
    if (t_ref) *t_ref = cv.t_ref;
    if (period_min) *period_min = cv.pmin;
    if (period_ratio) *period_ratio = cv.ratio;
    if (n_periods) *n_periods = cv.n_periods;
    if (n_t0) *n_t0 = cv.I;
    if (first_item) *first_item = b->group_off[curve];
    return CETRA_OK;
}

int cetra_batch_get_info(const cetra_batch *b, cetra_batch_info *info) {
    if (!b || !info) return CETRA_EINVAL;
    info->n_curves = b->n_curves;
    info->n_dur = b->plan->J;
    info->n_points = b->n_points;
    info->n_cells = b->n_cells;
    info->n_t0 = b->n_t0;
    info->n_periods = b->n_periods;
    info->n_fold_items = b->n_items;
    info->fold_cell_reads = b->fold_cell_reads;
    info->device_bytes = b->d_bytes;
    info->linear_threads = b->lin_threads;
    info->fold_variant = b->fold_variant;
    info->fold_blocks = b->fold_blocks;
    info->graph = b->graph != nullptr;
    info->cadence = b->plan->cadence;
    info->t0_step = b->plan->t0_step;
    info->p = b->plan->p;
    info->q = b->plan->q;
    info->n_pad = b->plan->n_pad;
    return CETRA_OK;
}

void cetra_batch_destroy(cetra_batch *b) {
    if (!b) return;
    device_guard dguard(b->device);
    release(b);
}

int cetra_search_batch(cetra_ctx *ctx, const cetra_params *params, int n_curves,
                       const int64_t *offsets, const double *time, const float *flux,
                       const float *flux_err, const double *durations, int n_dur,
                       const float *tmpl, int tmpl_len, const double *period_min,
                       const double *period_max, const double *period_ratio, cetra_best *best) {
    cetra_batch *b = nullptr;
    int rc = cetra_batch_create(ctx, params, n_curves, offsets, time, flux, flux_err, durations,
                                n_dur, tmpl, tmpl_len, period_min, period_max, period_ratio, 0, &b);
    if (rc) return rc;
    rc = cetra_batch_run(ctx, b, best);
    cetra_batch_destroy(b);
    return rc;
}

}  // extern "C"
