// The periodic search of a batch of light curves (Sec. 2.3, many curves per launch):
// batch_fold_kernel and its launcher. The device code it shares with the single-curve
// fold is in fold.cuh.
#include "fold.cuh"

namespace {

// Batched form: persistent blocks drain a queue of (curve, group of FT_G periods) items; each
// group's best per period goes into the curve's key (LR bits, inverted period index: the
// largest LR wins, ties to the smallest period index).
// Queue order (item_list NULL): the curves in the order order_curve[] (largest first), each
// curve's groups from its longest periods down, so that the last items of the queue are the
// cheapest; order_off is the prefix count of items over that order.
template <bool KAHAN, int R>
__global__ void __launch_bounds__(FT_BLOCK, FT_MIN_BLOCKS)
batch_fold_kernel(const float2 *__restrict__ ab, const batch_curve *__restrict__ curves,
                  const int64_t *__restrict__ group_off, int n_curves, int64_t n_items, int J,
                  const double *__restrict__ durations, double c, int64_t p, int64_t q,
                  int *__restrict__ queue, unsigned long long *__restrict__ period_keys,
                  unsigned long long *__restrict__ curve_keys, int *__restrict__ status,
                  const int64_t *__restrict__ item_list,
                  const unsigned long long *__restrict__ n_items_dev,
                  const int64_t *__restrict__ order_off, const int32_t *__restrict__ order_curve,
                  int gmax) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ fold_smem sm;
    __shared__ int s_item;
    // the queue length: n_items, or the count a device-side selection left (capped by n_items)
    if (n_items_dev) n_items = min(n_items, (int64_t)*n_items_dev);
    unsigned char *tab;
    best_slots bs;
    fold_smem_views(smem_raw, tab, bs);
    const int t = threadIdx.x;
    fold_init_barriers(sm);
    ring rg;
    for (;;) {
        block_sync();  // the previous item is done with the shared state
        if (t == 0) s_item = atomicAdd(queue, 1);
        block_sync();
        if (s_item >= n_items) break;
        // queue position -> work item: the caller's list entry, or the position in the order
        int64_t item;
        if (item_list) {
            item = item_list[s_item];
        } else {
            const int oc = csr_find(order_off, n_curves, (int64_t)s_item);
            const int cc = order_curve[oc];
            item = group_off[cc] + (order_off[oc + 1] - 1 - (int64_t)s_item);
        }
        const int cidx = csr_find(group_off, n_curves, item);
        const batch_curve cv = curves[cidx];
        const int k0 = (int)(item - group_off[cidx]) * FT_G;
        if (t == 0) {
            sm.it.ab = ab + cv.ab_off;
            sm.it.durations = durations;
            sm.it.mask = nullptr;
            sm.it.status = status;
            sm.it.ld = cv.ld;
            sm.it.I = cv.I;
            sm.it.J = J;
            sm.it.jlo = 0;
            sm.it.jhi = J;
            sm.it.mask_k0 = 0;
            sm.it.gmax = gmax;
        }
        if (t < FT_G) {
            const bool present = k0 + t < cv.n_periods;
            fold_slot_meta(sm, t, present, present ? batch_period(cv.pmin, cv.ratio, k0 + t) : 0.0,
                           cv.I, c, p, q);
        }
        block_sync();
        fold_group<KAHAN, R>(sm, smem_raw, tab, bs, rg);
        block_sync();
        if (sm.abort) {
            drain_copies(sm, rg);
            return;
        }
        if (t < FT_G && k0 + t < cv.n_periods) {
            const unsigned long long v = sm.best[t];
            period_keys[cv.per_off + k0 + t] = v;
            if (v != 0ull)
                atomicMax(&curve_keys[cidx], (v & 0xFFFFFFFF00000000ull) |
                                                 (unsigned long long)(0xFFFFFFFFu - (uint32_t)(k0 + t)));
        }
    }
}

}  // namespace

cudaError_t batch_fold_configure() {
    const int bytes = (int)fold_smem_bytes();
    for (auto fn : {batch_fold_kernel<false, FT_R>, batch_fold_kernel<false, FT_R / 2>,
                    batch_fold_kernel<true, FT_R / 2>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Fold variants the autotuner chooses from: bit 0 set = FT_R / 2 phases per thread (else
// FT_R), bit 1 set = sub-groups of at most FT_G / 2 periods (else FT_G). The compensated form
// always takes FT_R / 2 phases per thread.
int batch_fold_variants() { return 4; }
int batch_fold_blocks_per_sm(int) { return FT_MIN_BLOCKS; }

cudaError_t launch_batch_fold(cudaStream_t stream, int blocks, int variant, const cetra_plan *plan,
                              const float2 *ab, const batch_curve *curves,
                              const int64_t *group_off, int n_curves, int64_t n_items,
                              int *queue, unsigned long long *period_keys,
                              unsigned long long *curve_keys, int *status,
                              const int64_t *item_list, const unsigned long long *n_items_dev,
                              const int64_t *order_off, const int32_t *order_curve) {
    if (n_items <= 0) return cudaSuccess;
    auto kern = batch_fold_kernel<false, FT_R>;
    if (plan->precision == CETRA_FP32_KAHAN)
        kern = batch_fold_kernel<true, FT_R / 2>;
    else if (variant & 1)
        kern = batch_fold_kernel<false, FT_R / 2>;
    const int gmax = (variant & 2) ? FT_G / 2 : FT_G;
    kern<<<blocks, FT_BLOCK, fold_smem_bytes(), stream>>>(
        ab, curves, group_off, n_curves, n_items, plan->J, plan->d_durations, plan->cadence,
        plan->p, plan->q, queue, period_keys, curve_keys, status, item_list, n_items_dev,
        order_off, order_curve, gmax);
    return cudaGetLastError();
}
