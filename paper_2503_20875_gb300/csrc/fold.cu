// The periodic search of one light curve (Sec. 2.3): fold_kernel and its launcher. The
// device code it shares with the batched form is in fold.cuh.
#include <algorithm>

#include "fold.cuh"

namespace {

// Single light curve. Work item = (duration chunk, group); chunks outermost so that the blocks
// running at the same time read the same grid rows; within a chunk the groups run from the
// last (the longest periods of an ascending grid: the most phases, the most work) to the first.
// accumulate = 1: several chunks per period, keys combined with atomicMax (zeroed before).
template <bool KAHAN>
__global__ void __launch_bounds__(FT_BLOCK, FT_MIN_BLOCKS)
fold_kernel(const float2 *__restrict__ ab, int I, int64_t ld, int J,
            const double *__restrict__ durations, const double *__restrict__ periods, int K,
            const uint8_t *__restrict__ mask, double c, int64_t p, int64_t q, int n_groups,
            int jchunk, int accumulate, unsigned long long *__restrict__ keys,
            int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ fold_smem sm;
    unsigned char *tab;
    best_slots bs;
    fold_smem_views(smem_raw, tab, bs);
    const int t = threadIdx.x;
    const int jc = blockIdx.x / n_groups;
    const int grp = n_groups - 1 - (int)(blockIdx.x % n_groups);
    const int k0 = grp * FT_G;
    fold_init_barriers(sm);
    if (t == 0) {
        sm.it.ab = ab;
        sm.it.durations = durations;
        sm.it.mask = mask;
        sm.it.status = status;
        sm.it.ld = ld;
        sm.it.I = I;
        sm.it.J = J;
        sm.it.jlo = jc * jchunk;
        sm.it.jhi = min(J, sm.it.jlo + jchunk);
        sm.it.mask_k0 = k0;
        sm.it.gmax = FT_G;
    }
    if (t < FT_G) fold_slot_meta(sm, t, k0 + t < K, k0 + t < K ? periods[k0 + t] : 0.0, I, c, p, q);
    block_sync();
    ring rg;
    constexpr int R = KAHAN ? FT_R / 2 : FT_R;
    fold_group<KAHAN, R>(sm, smem_raw, tab, bs, rg);
    block_sync();
    if (sm.abort) {
        drain_copies(sm, rg);
        return;
    }
    if (t < FT_G && k0 + t < K) {
        const unsigned long long v = sm.best[t];
        if (!accumulate)
            keys[k0 + t] = v;
        else if (v)
            atomicMax(&keys[k0 + t], v);
    }
}

}  // namespace

size_t fold_smem_bytes() {
    return (size_t)FT_RING_BYTES + (size_t)FT_TAB_BYTES +
           (size_t)FT_G * FT_THREADS * (sizeof(float) + sizeof(uint32_t));
}
cudaError_t fold_configure() {
    const int bytes = (int)fold_smem_bytes();
    for (auto fn : {fold_kernel<false>, fold_kernel<true>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return batch_fold_configure();
}

cudaError_t launch_fold(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                        const double *periods, int K, const uint8_t *mask,
                        unsigned long long *keys, int *status) {
    if (K <= 0) return cudaSuccess;
    const int n_groups = (K + FT_G - 1) / FT_G;
    const size_t grid_bytes = (size_t)plan->J * (size_t)plan->ab_ld * sizeof(float2);
    // one duration per work item when the grid exceeds the L2 (the blocks in flight then share
    // a row); when whole groups would not give every block slot of the GPU FT_ITEMS_PER_SLOT
    // items, the durations are split into chunks as long as that many items still result
    const int64_t slots = (int64_t)ctx->num_sms * FT_MIN_BLOCKS;
    int jchunk = plan->J;
    if (grid_bytes > FT_L2_GRID_BYTES)
        jchunk = 1;
    else if ((int64_t)n_groups < FT_ITEMS_PER_SLOT * slots)
        jchunk = (int)std::max<int64_t>(
            1, (int64_t)n_groups * plan->J / ((int64_t)FT_ITEMS_PER_SLOT * slots));
    const int n_chunks = (plan->J + jchunk - 1) / jchunk;
    const int64_t items = (int64_t)n_groups * n_chunks;
    if (items > 2147483647) return cudaErrorInvalidConfiguration;
    const int accumulate = n_chunks > 1;
    if (accumulate) {
        cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)K * sizeof(unsigned long long), ctx->stream);
        if (e != cudaSuccess) return e;
    }
    prof_mark(ctx, KID_FOLD, true);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? fold_kernel<true> : fold_kernel<false>;
    kern<<<(unsigned)items, FT_BLOCK, fold_smem_bytes(), ctx->stream>>>(
        ab, (int)plan->n_t0, plan->ab_ld, plan->J, plan->d_durations, periods, K, mask,
        plan->cadence, plan->p, plan->q, n_groups, jchunk, accumulate, keys, status);
    prof_mark(ctx, KID_FOLD, false);
    ctx->launches++;
    return cudaGetLastError();
}
