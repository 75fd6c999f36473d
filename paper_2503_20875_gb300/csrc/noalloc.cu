// cetra_periodic_device_static: the periodic stage with its scratch in a static
// device array, for callers that cannot allocate device memory.
//
// The ordinary cetra_periodic_device needs a workspace sized for the number of
// periods: the fold writes one 64-bit key per period and a status word there
// before the finalize kernel reads them. Some callers cannot provide that: a
// caller that owns a fixed pool and may not call cudaMalloc while it runs, a
// plugin that receives device buffers from a host application with its own
// allocator, or a pipeline that sizes its workspace once for the linear grid and
// then sweeps period grids of varying length. This entry point keeps those keys
// and the status word in `g_fold_scratch` below instead, so the caller passes
// only the linear grid it already has, the periods and the output arrays.
//
// The array holds CETRA_STATIC_MAX_PERIODS keys plus the status word (2 MiB +
// 256 B). Every GPU that loads the library holds its own copy until the process
// exits. All calls on one device share it: calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it and must be
// serialised by the caller. Each call clears the status word before its fold
// runs. The keys are cleared only when the fold splits a period's durations over
// several blocks (it then zeroes them and combines the blocks' keys by atomic max);
// otherwise every block of a fold that completes writes the keys of all its
// periods before the finalize kernel reads them, and in both cases a block whose
// bounded wait gives up stops without writing its keys but first records
// CETRA_ETIMEOUT in the status word. The finalize kernel reads the status word
// first and writes NaN for every period when it is non-zero, so keys left over
// from an earlier call are never used. cetra_static_status reads the status word
// back.
#include "internal.h"

namespace {

constexpr int kStaticMaxPeriods = CETRA_STATIC_MAX_PERIODS;
constexpr size_t kKeysBytes = (size_t)kStaticMaxPeriods * sizeof(unsigned long long);

// Keys of the fold (one per period), then the status word at kKeysBytes.
static __device__ __align__(256) unsigned char g_fold_scratch[kKeysBytes + 256];

// The host-side name g_fold_scratch is only a stand-in for the symbol: its device
// address is looked up with the context's device current. The lookup is repeated on
// every call (it allocates nothing), so an address never outlives the device context
// it belongs to (a cudaDeviceReset by the host application re-creates it).
int scratch_address(cetra_ctx *ctx, const char *who, unsigned long long **keys, int **status) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fold_scratch);
    if (e != cudaSuccess || !p)
        return set_error(ctx, CETRA_ECUDA,
                         std::string(who) + ": scratch address: " + cudaGetErrorString(e));
    *keys = static_cast<unsigned long long *>(p);
    *status = reinterpret_cast<int *>(static_cast<char *>(p) + kKeysBytes);
    return CETRA_OK;
}

}  // namespace

extern "C" int cetra_periodic_device_static(cetra_ctx *ctx, const cetra_plan *plan,
                                            void *d_workspace, size_t workspace_bytes,
                                            const double *d_periods, int n_periods,
                                            const uint8_t *d_mask, double *d_dlogl, double *d_t0,
                                            double *d_duration, double *d_depth,
                                            double *d_depth_var, int64_t *d_i, int32_t *d_j) {
    if (!ctx || !plan || !d_workspace)
        return set_error(ctx, CETRA_EINVAL, "periodic_device_static: NULL argument");
    if (n_periods < 0)
        return set_error(ctx, CETRA_EINVAL, "periodic_device_static: n_periods < 0");
    if (n_periods > kStaticMaxPeriods)
        return set_error(ctx, CETRA_ECAPACITY,
                         "periodic_device_static: n_periods exceeds the static scratch limit of " +
                             std::to_string(kStaticMaxPeriods) + " periods");
    if (n_periods == 0) return CETRA_OK;
    if (!d_periods) return set_error(ctx, CETRA_EINVAL, "periodic_device_static: NULL periods");
    // only the linear grid is needed in the caller's workspace: keys live in the static array
    const ws_layout L = workspace_layout(plan, 0);
    if (workspace_bytes < L.total)
        return set_error(ctx, CETRA_ECAPACITY, "periodic_device_static: workspace too small");
    device_guard guard(ctx->device);
    if (guard.status != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA, std::string("periodic_device_static: device: ") +
                                               cudaGetErrorString(guard.status));
    unsigned long long *keys = nullptr;
    int *status = nullptr;
    int rc = scratch_address(ctx, "periodic_device_static", &keys, &status);
    if (rc != CETRA_OK) return rc;
    const float2 *ab = reinterpret_cast<const float2 *>(static_cast<char *>(d_workspace) + L.ab);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA,
                         std::string("periodic_device_static: status clear: ") + cudaGetErrorString(e));
    e = launch_fold(ctx, plan, ab, d_periods, n_periods, d_mask, keys, status);
    if (e != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA,
                         std::string("periodic_device_static: fold launch: ") + cudaGetErrorString(e));
    e = launch_finalize(ctx, plan, ab, d_periods, n_periods, keys, status, d_dlogl, d_t0,
                        d_duration, d_depth, d_depth_var, d_i, d_j);
    if (e != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA, std::string("periodic_device_static: finalize launch: ") +
                                               cudaGetErrorString(e));
    return CETRA_OK;
}

extern "C" int cetra_static_status(cetra_ctx *ctx, int *status) {
    if (!ctx || !status) return set_error(ctx, CETRA_EINVAL, "static_status: NULL argument");
    device_guard guard(ctx->device);
    if (guard.status != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA,
                         std::string("static_status: device: ") + cudaGetErrorString(guard.status));
    unsigned long long *keys = nullptr;
    int *d_status = nullptr;
    int rc = scratch_address(ctx, "static_status", &keys, &d_status);
    if (rc != CETRA_OK) return rc;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA,
                         std::string("static_status: read: ") + cudaGetErrorString(e));
    *status = h;
    return CETRA_OK;
}

extern "C" int cetra_selftest_static_timeout(cetra_ctx *ctx) {
    if (!ctx) return set_error(ctx, CETRA_EINVAL, "selftest_static_timeout: NULL context");
    device_guard guard(ctx->device);
    if (guard.status != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA, std::string("selftest_static_timeout: device: ") +
                                               cudaGetErrorString(guard.status));
    unsigned long long *keys = nullptr;
    int *status = nullptr;
    int rc = scratch_address(ctx, "selftest_static_timeout", &keys, &status);
    if (rc != CETRA_OK) return rc;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_wait_timeout_selftest(ctx->stream, nullptr, status);
    if (e != cudaSuccess)
        return set_error(ctx, CETRA_ECUDA,
                         std::string("selftest_static_timeout: ") + cudaGetErrorString(e));
    ctx->launches++;
    return CETRA_OK;
}
