// C ABI of the CETRA library (declarations and contracts in include/cetra.h).
// Argument checking, workspace layout, stream-ordered launches and the
// host-buffer convenience API. No compute happens here: every stage of the
// search runs in the kernels of kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

int set_error(cetra_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

const char *const kernel_names[KID_COUNT] = {"resample", "linear", "fold", "finalize", "logl0"};

namespace {
cudaEvent_t pool_event(cetra_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

void prof_mark(cetra_ctx *ctx, kernel_id id, bool begin) {
    if (!ctx->profiling) return;
    if (begin) {
        cudaEvent_t a = pool_event(ctx);
        if (!a) return;
        cudaEventRecord(a, ctx->stream);
        ctx->pending[id].push_back({a, nullptr});
    } else {
        if (ctx->pending[id].empty() || ctx->pending[id].back().second) return;
        cudaEvent_t b = pool_event(ctx);
        if (!b) return;
        cudaEventRecord(b, ctx->stream);
        ctx->pending[id].back().second = b;
    }
}

namespace {

int cuda_fail(cetra_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, CETRA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The three device regions of a workspace.
struct ws_ptrs {
    float2 *grid;  // interleaved (W y, W)
    int *lin_status;
    float2 *ab;
    unsigned long long *keys;
    double *logl0;
    int *status;
};

ws_ptrs carve(void *base, const ws_layout &L) {
    char *b = static_cast<char *>(base);
    return ws_ptrs{reinterpret_cast<float2 *>(b + L.grid), reinterpret_cast<int *>(b + L.lin_status),
                   reinterpret_cast<float2 *>(b + L.ab),
                   reinterpret_cast<unsigned long long *>(b + L.keys),
                   reinterpret_cast<double *>(b + L.logl0), reinterpret_cast<int *>(b + L.status)};
}

void fill_info(const cetra_plan *plan, cetra_plan_info *info) {
    info->t_ref = plan->t_ref;
    info->cadence = plan->cadence;
    info->t0_step = plan->t0_step;
    info->p = plan->p;
    info->q = plan->q;
    info->n_pad = plan->n_pad;
    info->n_grid = plan->n_grid;
    info->n_t0 = plan->n_t0;
    info->n_kept = plan->n_kept;
    info->n_dur = plan->J;
    info->template_samples = plan->L;
    info->table_entries = (int64_t)plan->tables.size();
    info->grid_bytes = workspace_layout(plan, 0).total;
}

}  // namespace

extern "C" {

void cetra_params_default(cetra_params *p) {
    if (!p) return;
    p->cadence = 0.0;
    p->t0_step = 0.0;
    p->template_samples = 1024;
    p->flux_is_offset = 0;
    p->precision = CETRA_FP32;
}

int cetra_create(cetra_ctx **out, int device, void *cuda_stream) {
    if (!out) return CETRA_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return CETRA_ECUDA;
    }
    cetra_ctx *ctx = new (std::nothrow) cetra_ctx;
    if (!ctx) return CETRA_ENOMEM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    device_guard g(device);
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) == cudaSuccess)
        ctx->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) == cudaSuccess)
        ctx->max_smem_optin = (size_t)v;
    if (ctx->num_sms <= 0) ctx->num_sms = 1;
    *out = ctx;
    return CETRA_OK;
}

void cetra_destroy(cetra_ctx *ctx) {
    if (!ctx) return;
    {
        device_guard g(ctx->device);
        for (auto &v : ctx->pending)
            for (auto &pr : v) {
                if (pr.first) cudaEventDestroy(pr.first);
                if (pr.second) cudaEventDestroy(pr.second);
            }
        for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    }
    delete ctx;
}

int cetra_profile_enable(cetra_ctx *ctx, int enable) {
    if (!ctx) return CETRA_EINVAL;
    ctx->profiling = enable != 0;
    return CETRA_OK;
}

int cetra_profile_read(cetra_ctx *ctx, const char *kernel, int64_t *launches, double *total_ms) {
    if (!ctx || !kernel) return set_error(ctx, CETRA_EINVAL, "profile_read: NULL argument");
    int id = -1;
    for (int k = 0; k < KID_COUNT; ++k)
        if (std::strcmp(kernel, kernel_names[k]) == 0) id = k;
    if (id < 0) return set_error(ctx, CETRA_EINVAL, std::string("profile_read: unknown kernel ") + kernel);
    device_guard g(ctx->device);
    double sum = 0.0;
    int64_t n = 0;
    for (auto &pr : ctx->pending[id]) {
        if (pr.second) {
            if (cudaEventSynchronize(pr.second) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "profile_read");
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
                sum += ms;
                ++n;
            }
            ctx->event_pool.push_back(pr.second);
        }
        ctx->event_pool.push_back(pr.first);
    }
    ctx->pending[id].clear();
    if (launches) *launches = n;
    if (total_ms) *total_ms = sum;
    return CETRA_OK;
}

int cetra_set_stream(cetra_ctx *ctx, void *cuda_stream) {
    if (!ctx) return CETRA_EINVAL;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return CETRA_OK;
}

const char *cetra_last_error(const cetra_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int64_t cetra_kernel_launches(const cetra_ctx *ctx) { return ctx ? ctx->launches : 0; }

int cetra_plan_create(cetra_ctx *ctx, const cetra_params *params, const double *time,
                      const float *flux, const float *flux_err, int64_t n_points,
                      const double *durations, int n_dur, const float *tmpl, int tmpl_len,
                      cetra_plan **plan_out) {
    if (!ctx || !plan_out) return set_error(ctx, CETRA_EINVAL, "plan: NULL ctx or plan");
    *plan_out = nullptr;
    cetra_params def;
    cetra_params_default(&def);
    if (!params) params = &def;
    if (params->precision != CETRA_FP32 && params->precision != CETRA_FP32_KAHAN)
        return set_error(ctx, CETRA_EINVAL, "plan: unknown precision");
    device_guard g(ctx->device);
    cetra_plan *plan = new (std::nothrow) cetra_plan;
    if (!plan) return set_error(ctx, CETRA_ENOMEM, "plan: host allocation");
    plan->device = ctx->device;
    int rc = plan_build(ctx, params, time, flux, flux_err, n_points, durations, n_dur, tmpl,
                        tmpl_len, plan, true);
    if (rc == CETRA_OK && (int64_t)plan->J * plan->q > 65535)
        rc = set_error(ctx, CETRA_EINVAL, "plan: n_dur * q exceeds 65535");
    if (rc == CETRA_OK) rc = plan_upload(ctx, plan);
    if (rc != CETRA_OK) {
        plan_free_device(plan);
        delete plan;
        return rc;
    }
    *plan_out = plan;
    return CETRA_OK;
}

int cetra_plan_geometry(cetra_ctx *ctx, const cetra_params *params, const double *time,
                        const float *flux, const float *flux_err, int64_t n_points,
                        const double *durations, int n_dur, cetra_plan_info *info) {
    if (!info) return set_error(ctx, CETRA_EINVAL, "geometry: NULL info");
    cetra_params def;
    cetra_params_default(&def);
    if (!params) params = &def;
    cetra_plan plan;
    int rc = plan_build(ctx, params, time, flux, flux_err, n_points, durations, n_dur, nullptr, 0,
                        &plan, false);
    if (rc != CETRA_OK) return rc;
    fill_info(&plan, info);
    return CETRA_OK;
}

int cetra_plan_get_info(const cetra_plan *plan, cetra_plan_info *info) {
    if (!plan || !info) return CETRA_EINVAL;
    fill_info(plan, info);
    return CETRA_OK;
}

void cetra_plan_destroy(cetra_plan *plan) {
    if (!plan) return;
    device_guard g(plan->device);
    plan_free_device(plan);
    delete plan;
}

size_t cetra_workspace_bytes(const cetra_plan *plan, int n_periods) {
    return plan ? workspace_layout(plan, n_periods).total : 0;
}

int cetra_resample_device(cetra_ctx *ctx, const cetra_plan *plan, const double *d_time,
                          const float *d_flux, const float *d_flux_err, int64_t n_points,
                          void *d_workspace, size_t workspace_bytes) {
    if (!ctx || !plan || !d_workspace) return set_error(ctx, CETRA_EINVAL, "resample: NULL argument");
    if (n_points < 0) return set_error(ctx, CETRA_EINVAL, "resample: n_points < 0");
    if (n_points > 0 && (!d_time || !d_flux || !d_flux_err))
        return set_error(ctx, CETRA_EINVAL, "resample: NULL input array");
    ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "resample: workspace too small");
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    cudaError_t e = cudaMemsetAsync(w.grid, 0, L.ab - L.grid, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "resample memset");
    e = launch_resample(ctx, plan, d_time, d_flux, d_flux_err, n_points, w.grid);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "resample launch");
    return CETRA_OK;
}

int cetra_linear_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                        size_t workspace_bytes, float *d_depth, float *d_depth_var,
                        float *d_dlogl) {
    if (!ctx || !plan || !d_workspace) return set_error(ctx, CETRA_EINVAL, "linear: NULL argument");
    ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "linear: workspace too small");
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    // the zero cells after each grid row, read by the fold's bulk copies
    const size_t pitch = (size_t)plan->ab_ld * sizeof(float2);
    cudaError_t e = cudaMemset2DAsync(w.ab + plan->n_t0, pitch, 0,
                                      (size_t)(plan->ab_ld - plan->n_t0) * sizeof(float2),
                                      (size_t)plan->J, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "linear padding memset");
    e = cudaMemsetAsync(w.lin_status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "linear status memset");
    e = launch_linear(ctx, plan, w.grid, w.ab, d_depth, d_depth_var, d_dlogl, w.lin_status);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "linear launch");
    return CETRA_OK;
}

int cetra_periodic_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                          size_t workspace_bytes, const double *d_periods, int n_periods,
                          const uint8_t *d_mask, double *d_dlogl, double *d_t0,
                          double *d_duration, double *d_depth, double *d_depth_var,
                          int64_t *d_i, int32_t *d_j) {
    if (!ctx || !plan || !d_workspace) return set_error(ctx, CETRA_EINVAL, "periodic: NULL argument");
    if (n_periods < 0) return set_error(ctx, CETRA_EINVAL, "periodic: n_periods < 0");
    if (n_periods == 0) return CETRA_OK;
    if (!d_periods) return set_error(ctx, CETRA_EINVAL, "periodic: NULL periods");
    ws_layout L = workspace_layout(plan, n_periods);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "periodic: workspace too small");
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "periodic status memset");
    e = launch_fold(ctx, plan, w.ab, d_periods, n_periods, d_mask, w.keys, w.status);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fold launch");
    e = launch_finalize(ctx, plan, w.ab, d_periods, n_periods, w.keys, w.status, d_dlogl, d_t0,
                        d_duration, d_depth, d_depth_var, d_i, d_j);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "finalize launch");
    return CETRA_OK;
}

int cetra_workspace_status(cetra_ctx *ctx, const cetra_plan *plan, const void *d_workspace,
                           size_t workspace_bytes, int *status) {
    if (!ctx || !plan || !d_workspace || !status)
        return set_error(ctx, CETRA_EINVAL, "workspace_status: NULL argument");
    ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "workspace_status: workspace too small");
    device_guard g(ctx->device);
    int v = 0, vl = 0;
    cudaError_t e = cudaMemcpyAsync(&v, static_cast<const char *>(d_workspace) + L.status,
                                    sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&vl, static_cast<const char *>(d_workspace) + L.lin_status,
                            sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace_status");
    *status = v ? v : vl;  // the periodic stage's word, else the linear stage's
    return CETRA_OK;
}

int cetra_logl0_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                       size_t workspace_bytes, double *d_logl0) {
    if (!ctx || !plan || !d_workspace || !d_logl0)
        return set_error(ctx, CETRA_EINVAL, "logl0: NULL argument");
    ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "logl0: workspace too small");
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    cudaError_t e = launch_logl0(ctx, plan, w.grid, d_logl0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "logl0 launch");
    return CETRA_OK;
}

// ------------------------------------------------------------------------------ host-buffer API

int cetra_linear_search(cetra_ctx *ctx, const cetra_params *params, const double *time,
                        const float *flux, const float *flux_err, int64_t n_points,
                        const double *durations, int n_dur, const float *tmpl, int tmpl_len,
                        cetra_linear_grid **grid_out, float *depth, float *depth_var,
                        float *dlogl, int64_t *n_t0) {
    if (!ctx) return CETRA_EINVAL;
    if (grid_out) *grid_out = nullptr;
    if ((depth || depth_var || dlogl) && !n_t0)
        return set_error(ctx, CETRA_EINVAL, "linear_search: n_t0 capacity required with outputs");
    cetra_plan *plan = nullptr;
    int rc = cetra_plan_create(ctx, params, time, flux, flux_err, n_points, durations, n_dur, tmpl,
                               tmpl_len, &plan);
    if (rc) return rc;
    const int64_t I = plan->n_t0;
    if ((depth || depth_var || dlogl) && *n_t0 < I) {
        *n_t0 = I;
        cetra_plan_destroy(plan);
        return set_error(ctx, CETRA_ECAPACITY, "linear_search: output capacity below n_t0");
    }
    if (n_t0) *n_t0 = I;
    device_guard g(ctx->device);
    cetra_linear_grid *grid = new (std::nothrow) cetra_linear_grid;
    if (!grid) {
        cetra_plan_destroy(plan);
        return set_error(ctx, CETRA_ENOMEM, "linear_search: host allocation");
    }
    grid->ctx = ctx;
    grid->plan = plan;
    grid->work_bytes = workspace_layout(plan, 0).total;
    auto fail = [&](int code) {
        cetra_grid_free(grid);
        return code;
    };
    cudaError_t e = cudaMalloc(&grid->d_work, grid->work_bytes);
    if (e != cudaSuccess) {
        grid->d_work = nullptr;
        return fail(set_error(ctx, CETRA_ENOMEM, "linear_search: workspace allocation"));
    }
    // inputs
    const size_t nb_t = (size_t)n_points * sizeof(double), nb_f = (size_t)n_points * sizeof(float);
    void *d_in = nullptr;
    e = cudaMalloc(&d_in, nb_t + 2 * nb_f + 64);
    if (e != cudaSuccess) return fail(set_error(ctx, CETRA_ENOMEM, "linear_search: input allocation"));
    double *d_t = static_cast<double *>(d_in);
    float *d_f = reinterpret_cast<float *>(static_cast<char *>(d_in) + nb_t);
    float *d_e = d_f + n_points;
    cudaError_t ce = cudaMemcpyAsync(d_t, time, nb_t, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_f, flux, nb_f, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_e, flux_err, nb_f, cudaMemcpyHostToDevice, ctx->stream);
    rc = ce != cudaSuccess ? cuda_fail(ctx, ce, "linear_search: input copy")
                           : cetra_resample_device(ctx, plan, d_t, d_f, d_e, n_points,
                                                   grid->d_work, grid->work_bytes);
    float *d_out = nullptr;
    const size_t cells = (size_t)plan->J * (size_t)I;
    int nout = (depth ? 1 : 0) + (depth_var ? 1 : 0) + (dlogl ? 1 : 0);
    if (rc == CETRA_OK && nout) {
        e = cudaMalloc((void **)&d_out, cells * sizeof(float) * nout);
        if (e != cudaSuccess) rc = set_error(ctx, CETRA_ENOMEM, "linear_search: output allocation");
    }
    if (rc == CETRA_OK) {
        float *o = d_out;
        float *dd = depth ? o : nullptr;
        if (depth) o += cells;
        float *dv = depth_var ? o : nullptr;
        if (depth_var) o += cells;
        float *dl = dlogl ? o : nullptr;
        rc = cetra_linear_device(ctx, plan, grid->d_work, grid->work_bytes, dd, dv, dl);
        if (rc == CETRA_OK) {
            if (depth) ce = cudaMemcpyAsync(depth, dd, cells * 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (depth_var && ce == cudaSuccess)
                ce = cudaMemcpyAsync(depth_var, dv, cells * 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (dlogl && ce == cudaSuccess)
                ce = cudaMemcpyAsync(dlogl, dl, cells * 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "linear_search: output copy");
        }
    }
    e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_in);
    cudaFree(d_out);
    if (rc != CETRA_OK) return fail(rc);
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "linear_search"));
    if (grid_out)
        *grid_out = grid;
    else
        cetra_grid_free(grid);
    return CETRA_OK;
}

namespace {
// Enlarge a grid's workspace to `total` bytes, keeping its contents.
int grow_workspace(cetra_ctx *ctx, cetra_linear_grid *grid, size_t total) {
    if (grid->work_bytes >= total) return CETRA_OK;
    void *bigger = nullptr;
    cudaError_t e = cudaMalloc(&bigger, total);
    if (e != cudaSuccess) return set_error(ctx, CETRA_ENOMEM, "workspace allocation");
    e = cudaMemcpyAsync(bigger, grid->d_work, grid->work_bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(bigger);
        return cuda_fail(ctx, e, "workspace copy");
    }
    cudaFree(grid->d_work);
    grid->d_work = bigger;
    grid->work_bytes = total;
    return CETRA_OK;
}
}  // namespace

int cetra_periodic_search(cetra_ctx *ctx, cetra_linear_grid *grid, const double *periods,
                          int n_periods, const uint8_t *dur_mask, double *dlogl, double *t0,
                          double *duration, double *depth, double *depth_var, int64_t *best_k) {
    if (!ctx || !grid || !grid->plan) return set_error(ctx, CETRA_EINVAL, "periodic_search: NULL grid");
    if (n_periods < 0 || (n_periods > 0 && !periods))
        return set_error(ctx, CETRA_EINVAL, "periodic_search: bad periods");
    for (int k = 0; k < n_periods; ++k)
        if (!(periods[k] > 0.0) || !std::isfinite(periods[k]))
            return set_error(ctx, CETRA_EINVAL, "periodic_search: periods must be finite and > 0");
    if (best_k) *best_k = -1;
    if (n_periods == 0) return CETRA_OK;
    cetra_plan *plan = grid->plan;
    device_guard g(ctx->device);
    // the grid workspace is sized without keys; periodic needs a larger one
    int rc0 = grow_workspace(ctx, grid, workspace_layout(plan, n_periods).total);
    if (rc0 != CETRA_OK) return rc0;
    const size_t K = (size_t)n_periods, J = (size_t)plan->J;
    const size_t bytes = K * sizeof(double) * 6 + K * J + 256;
    char *d_buf = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_buf, bytes);
    if (e != cudaSuccess) return set_error(ctx, CETRA_ENOMEM, "periodic_search: buffer allocation");
    double *d_P = reinterpret_cast<double *>(d_buf);
    double *d_out = d_P + K;  // 5 K doubles
    uint8_t *d_mask = dur_mask ? reinterpret_cast<uint8_t *>(d_out + 5 * K) : nullptr;
    cudaError_t ce = cudaMemcpyAsync(d_P, periods, K * sizeof(double), cudaMemcpyHostToDevice,
                                     ctx->stream);
    if (dur_mask && ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_mask, dur_mask, K * J, cudaMemcpyHostToDevice, ctx->stream);
    int rc = ce != cudaSuccess
                 ? cuda_fail(ctx, ce, "periodic_search: input copy")
                 : cetra_periodic_device(ctx, plan, grid->d_work, grid->work_bytes, d_P,
                                         n_periods, d_mask, d_out, d_out + K, d_out + 2 * K,
                                         d_out + 3 * K, d_out + 4 * K, nullptr, nullptr);
    double *h_lr = dlogl;
    std::vector<double> tmp;
    if (!h_lr && best_k) {
        tmp.resize(K);
        h_lr = tmp.data();
    }
    if (rc == CETRA_OK) {
        double *dst[5] = {h_lr, t0, duration, depth, depth_var};
        for (int m = 0; m < 5 && ce == cudaSuccess; ++m)
            if (dst[m])
                ce = cudaMemcpyAsync(dst[m], d_out + m * K, K * 8, cudaMemcpyDeviceToHost,
                                     ctx->stream);
        if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "periodic_search: output copy");
    }
    e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_buf);
    if (rc != CETRA_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "periodic_search");
    int st = 0;
    rc = cetra_workspace_status(ctx, plan, grid->d_work, grid->work_bytes, &st);
    if (rc != CETRA_OK) return rc;
    if (st != 0) return set_error(ctx, CETRA_ETIMEOUT, "periodic_search: a device wait timed out");
    if (best_k && h_lr) {
        int64_t bk = -1;
        double bv = -INFINITY;
        for (size_t k = 0; k < K; ++k)
            if (!std::isnan(h_lr[k]) && h_lr[k] > bv) {
                bv = h_lr[k];
                bk = (int64_t)k;
            }
        *best_k = bk;
    }
    return CETRA_OK;
}

int cetra_selftest_wait_timeout(cetra_ctx *ctx, int *timed_out, double *seconds) {
    if (!ctx || !timed_out) return set_error(ctx, CETRA_EINVAL, "selftest: NULL argument");
    device_guard g(ctx->device);
    int *d = nullptr;
    if (cudaMalloc((void **)&d, 2 * sizeof(int)) != cudaSuccess)
        return set_error(ctx, CETRA_ENOMEM, "selftest: allocation");
    int h[2] = {0, 0};
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    if (!e) e = cudaMemsetAsync(d, 0, 2 * sizeof(int), ctx->stream);
    if (!e) e = cudaEventRecord(a, ctx->stream);
    if (!e) e = launch_wait_timeout_selftest(ctx->stream, d);
    if (!e) e = cudaEventRecord(b, ctx->stream);
    if (!e) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    float ms = 0.0f;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(d);
    if (e) return cuda_fail(ctx, e, "selftest");
    ctx->launches++;
    *timed_out = h[0];
    if (seconds) *seconds = 1e-3 * ms;
    return CETRA_OK;
}

int cetra_measure_peaks(cetra_ctx *ctx, double *fma_tflops, double *smem_gbs) {
    if (!ctx) return set_error(ctx, CETRA_EINVAL, "measure_peaks: NULL context");
    device_guard g(ctx->device);
    const int grid[2] = {peak_grid(ctx->num_sms, false), peak_grid(ctx->num_sms, true)};
    const int iters[2] = {32768, 8192};  // a few ms a launch at the nominal rates
    float *d = nullptr;
    const size_t n = (size_t)std::max(grid[0], grid[1]) * PEAK_THREADS;
    if (cudaMalloc((void **)&d, n * sizeof(float)) != cudaSuccess)
        return set_error(ctx, CETRA_ENOMEM, "measure_peaks: allocation");
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    double rate[2] = {0.0, 0.0};
    for (int m = 0; m < 2 && !e; ++m) {
        double work = 0.0;
        e = launch_peak(ctx->stream, m == 1, grid[m], iters[m] / 8, d, &work);  // warm-up
        ctx->launches++;
        for (int rep = 0; rep < 3 && !e; ++rep) {
            e = cudaEventRecord(a, ctx->stream);
            if (!e) e = launch_peak(ctx->stream, m == 1, grid[m], iters[m], d, &work);
            if (!e) e = cudaEventRecord(b, ctx->stream);
            if (!e) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (!e) e = cudaEventElapsedTime(&ms, a, b);
            if (!e && ms > 0.0f) rate[m] = std::max(rate[m], work / (1e-3 * ms));
            ctx->launches++;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(d);
    if (e) return cuda_fail(ctx, e, "measure_peaks");
    if (fma_tflops) *fma_tflops = rate[0] * 1e-12;
    if (smem_gbs) *smem_gbs = rate[1] * 1e-9;
    return CETRA_OK;
}

// ------------------------------------------------------------------ method neighbours

int cetra_mask_transits_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                               size_t workspace_bytes, double period, double t0,
                               double half_width, unsigned long long *d_n_masked) {
    if (!ctx || !plan || !d_workspace) return set_error(ctx, CETRA_EINVAL, "mask: NULL argument");
    if (!(period > 0.0) || !std::isfinite(period) || !std::isfinite(t0) ||
        !(half_width >= 0.0) || !std::isfinite(half_width))
        return set_error(ctx, CETRA_EINVAL, "mask: period must be > 0, t0 and half_width finite, half_width >= 0");
    ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total) return set_error(ctx, CETRA_ECAPACITY, "mask: workspace too small");
    if (half_width == 0.0) return CETRA_OK;
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    cudaError_t e = launch_mask(ctx, plan, w.grid, period, t0, half_width, d_n_masked);
    return e != cudaSuccess ? cuda_fail(ctx, e, "mask launch") : CETRA_OK;
}

int cetra_mask_transits(cetra_ctx *ctx, cetra_linear_grid *grid, double period, double t0,
                        double half_width, int64_t *n_masked) {
    if (!ctx || !grid || !grid->plan) return set_error(ctx, CETRA_EINVAL, "mask_transits: NULL grid");
    device_guard g(ctx->device);
    unsigned long long *d_n = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_n, sizeof(unsigned long long));
    if (e != cudaSuccess) return set_error(ctx, CETRA_ENOMEM, "mask_transits: allocation");
    unsigned long long n = 0;
    e = cudaMemsetAsync(d_n, 0, sizeof(n), ctx->stream);
    int rc = e != cudaSuccess ? cuda_fail(ctx, e, "mask_transits") : CETRA_OK;
    if (rc == CETRA_OK)
        rc = cetra_mask_transits_device(ctx, grid->plan, grid->d_work, grid->work_bytes, period, t0,
                                        half_width, d_n);
    if (rc == CETRA_OK)  // the linear stage again, on the masked grid
        rc = cetra_linear_device(ctx, grid->plan, grid->d_work, grid->work_bytes, nullptr, nullptr,
                                 nullptr);
    if (rc == CETRA_OK) {
        e = cudaMemcpyAsync(&n, d_n, sizeof(n), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "mask_transits");
    }
    cudaFree(d_n);
    if (rc == CETRA_OK && n_masked) *n_masked = (int64_t)n;
    return rc;
}

int cetra_monotransits_device(cetra_ctx *ctx, const cetra_plan *plan, void *d_workspace,
                              size_t workspace_bytes, int max_events, cetra_event *d_events,
                              int *d_n_events) {
    if (!ctx || !plan || !d_workspace || !d_events || !d_n_events)
        return set_error(ctx, CETRA_EINVAL, "monotransits: NULL argument");
    if (max_events < 1 || max_events > CETRA_MAX_EVENTS)
        return set_error(ctx, CETRA_EINVAL, "monotransits: max_events outside 1..4096");
    if (plan->n_t0 > 0x1000000 || plan->J > 256)
        return set_error(ctx, CETRA_ECAPACITY, "monotransits: needs n_t0 <= 2^24 and n_dur <= 256");
    ws_layout L = workspace_layout(plan, (int)mono_scratch_words(plan, max_events));
    if (workspace_bytes < L.total)
        return set_error(ctx, CETRA_ECAPACITY, "monotransits: workspace too small");
    device_guard g(ctx->device);
    ws_ptrs w = carve(d_workspace, L);
    cudaError_t e = launch_monotransits(ctx, plan, w.ab, w.keys, max_events, d_events, d_n_events);
    return e != cudaSuccess ? cuda_fail(ctx, e, "monotransits launch") : CETRA_OK;
}

size_t cetra_monotransit_workspace_bytes(const cetra_plan *plan, int max_events) {
    if (!plan || max_events < 1) return 0;
    return workspace_layout(plan, (int)mono_scratch_words(plan, max_events)).total;
}

int cetra_monotransit_search(cetra_ctx *ctx, cetra_linear_grid *grid, int max_events,
                             cetra_event *events, int *n_events) {
    if (!ctx || !grid || !grid->plan || !events || !n_events)
        return set_error(ctx, CETRA_EINVAL, "monotransit_search: NULL argument");
    if (max_events < 1 || max_events > CETRA_MAX_EVENTS)
        return set_error(ctx, CETRA_EINVAL, "monotransit_search: max_events outside 1..4096");
    *n_events = 0;
    device_guard g(ctx->device);
    int rc = grow_workspace(ctx, grid, cetra_monotransit_workspace_bytes(grid->plan, max_events));
    if (rc != CETRA_OK) return rc;
    char *d_buf = nullptr;
    const size_t ev_bytes = (size_t)max_events * sizeof(cetra_event);
    cudaError_t e = cudaMalloc((void **)&d_buf, ev_bytes + 256);
    if (e != cudaSuccess) return set_error(ctx, CETRA_ENOMEM, "monotransit_search: allocation");
    cetra_event *d_ev = reinterpret_cast<cetra_event *>(d_buf);
    int *d_n = reinterpret_cast<int *>(d_buf + ev_bytes);
    rc = cetra_monotransits_device(ctx, grid->plan, grid->d_work, grid->work_bytes, max_events,
                                   d_ev, d_n);
    int n = 0;
    if (rc == CETRA_OK) {
        e = cudaMemcpyAsync(&n, d_n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(events, d_ev, ev_bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "monotransit_search");
    }
    cudaFree(d_buf);
    if (rc == CETRA_OK) *n_events = n;
    return rc;
}

int cetra_search_iterative(cetra_ctx *ctx, cetra_linear_grid *grid, const double *periods,
                           int n_periods, const uint8_t *dur_mask, int n_iter, double width,
                           cetra_best *out, int *n_found) {
    if (!ctx || !grid || !grid->plan || !out || !n_found)
        return set_error(ctx, CETRA_EINVAL, "search_iterative: NULL argument");
    if (n_iter < 1 || n_periods < 1 || !periods)
        return set_error(ctx, CETRA_EINVAL, "search_iterative: need n_iter >= 1 and periods");
    if (!(width > 0.0)) width = 2.0;
    if (!std::isfinite(width)) return set_error(ctx, CETRA_EINVAL, "search_iterative: width not finite");
    *n_found = 0;
    const size_t K = (size_t)n_periods;
    std::vector<double> lr(K), t0(K), dur(K), dep(K), var(K);
    for (int r = 0; r < n_iter; ++r) {
        int64_t bk = -1;
        int rc = cetra_periodic_search(ctx, grid, periods, n_periods, dur_mask, lr.data(),
                                       t0.data(), dur.data(), dep.data(), var.data(), &bk);
        if (rc != CETRA_OK) return rc;
        if (bk < 0) break;
        cetra_best b{};
        b.dlogl = lr[bk];
        b.period = periods[bk];
        b.t0 = t0[bk];
        b.duration = dur[bk];
        b.depth = dep[bk];
        b.depth_var = var[bk];
        b.k = bk;
        b.i = -1;
        b.j = -1;
        for (int j = 0; j < grid->plan->J; ++j)
            if (grid->plan->durations[j] == b.duration) {
                b.j = j;
                break;
            }
        b.n_periods = n_periods;
        out[r] = b;
        *n_found = r + 1;
        if (r + 1 < n_iter) {
            rc = cetra_mask_transits(ctx, grid, b.period, b.t0, 0.5 * width * b.duration, nullptr);
            if (rc != CETRA_OK) return rc;
        }
    }
    return CETRA_OK;
}

void cetra_grid_free(cetra_linear_grid *grid) {
    if (!grid) return;
    if (grid->plan) {
        device_guard g(grid->plan->device);
        cudaFree(grid->d_work);
    }
    cetra_plan_destroy(grid->plan);
    delete grid;
}

int cetra_grid_get_info(const cetra_linear_grid *grid, cetra_plan_info *info) {
    if (!grid || !grid->plan || !info) return CETRA_EINVAL;
    fill_info(grid->plan, info);
    return CETRA_OK;
}

}  // extern "C"
