// Method neighbours of the search (declarations in include/cetra.h):
//  - masking a detected signal before the next search (Sec. 4.2): the resampled cells in and
//    around the signal's transits are nulled, then the linear stage is rerun;
//  - single-transit (monotransit) events from the linear search (Sec. 1, Sec. 5): the
//    strongest dimming windows, greedily, each hiding the mid-times within its duration.
#include <cmath>

#include "internal.h"

namespace {

constexpr int NB_THREADS = 256;

// Null cell k (W y = W = 0) when its time g = t_ref + (k - n_pad) c is within h of a mid-time
// t0 + n P, n = floor((g - t0) / P + 1/2) the nearest epoch; FP64, one rounding per operation.
// counts[0] += cells that held data (counts may be NULL).
__global__ void mask_kernel(float2 *__restrict__ grid, int64_t n_grid,
                            double t_ref, double c, int64_t n_pad, double P, double t0, double h,
                            unsigned long long *__restrict__ counts) {
    unsigned long long mine = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_grid; k += stride) {
        const double g = __dadd_rn(t_ref, __dmul_rn((double)(k - n_pad), c));
        const double d = __dsub_rn(g, t0);
        const double n = floor(__dadd_rn(__ddiv_rn(d, P), 0.5));
        const double r = fabs(__dsub_rn(d, __dmul_rn(n, P)));
        if (r < h) {
            mine += grid[k].y > 0.0f;
            grid[k] = make_float2(0.0f, 0.0f);
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xFFFFFFFFu, mine, o);
    if (counts && (threadIdx.x & 31) == 0 && mine) atomicAdd(counts, mine);
}

// Event keys: per t0 cell the best dimming window over durations, packed so that a larger key
// is a better event: LR bits (positive floats order like their bits), then 255 - j (smaller j
// first), then 2^24 - 1 - i (smaller i first). 0 = no dimming window at this t0.
__device__ __forceinline__ unsigned long long event_key(float lr, int j, int64_t i) {
    return ((unsigned long long)__float_as_uint(lr) << 32) |
           ((unsigned long long)(255 - j) << 24) | (unsigned long long)(0xFFFFFF - i);
}

__global__ void mono_keys_kernel(const float2 *__restrict__ ab, int64_t ld, int64_t I, int J,
                                 unsigned long long *__restrict__ keys) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += stride) {
        unsigned long long best = 0ull;
        for (int j = 0; j < J; ++j) {
            const float2 v = ab[(int64_t)j * ld + i];
            if (v.y > 0.0f && v.x > 0.0f) {
                const float lr = 0.5f * (v.x * (v.x / v.y));
                if (lr > 0.0f) best = max(best, event_key(lr, j, i));
            }
        }
        keys[i] = best;
    }
}

// Greedy step e: the best key left (the cells earlier events hide have key 0). Nothing to do
// once a previous step found nothing.
__global__ void mono_pick_kernel(const unsigned long long *__restrict__ keys, int64_t I, int e,
                                 unsigned long long *__restrict__ slots) {
    if (e > 0 && slots[e - 1] == 0ull) return;  // uniform
    __shared__ unsigned long long red[NB_THREADS / 32];
    unsigned long long best = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += stride)
        best = max(best, keys[i]);
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int x = 1; x < NB_THREADS / 32; ++x) best = max(best, red[x]);
        if (best) atomicMax(&slots[e], best);
    }
}

// Decode step e's key into event e (FP64 values from the window's FP32 sums), then hide the
// t0 cells within its duration: |i - i_e| < h = D_j q / (c p) (FP64) -> key 0. One block.
__global__ void __launch_bounds__(NB_THREADS)
mono_event_kernel(const unsigned long long *__restrict__ slots, int e,
                  const float2 *__restrict__ ab, int64_t ld, int64_t I,
                  const double *__restrict__ durations, double t_ref, double c, int64_t p,
                  int64_t q, int64_t n_pad, unsigned long long *__restrict__ keys,
                  cetra_event *__restrict__ events, int *__restrict__ n_events) {
    const unsigned long long key = slots[e];
    if (key == 0ull || (e > 0 && slots[e - 1] == 0ull)) return;  // uniform
    const int64_t ie = 0xFFFFFF - (int64_t)(key & 0xFFFFFFull);
    const int j = 255 - (int)((key >> 24) & 0xFFull);
    const double h = __ddiv_rn(__dmul_rn(durations[j], (double)q), __dmul_rn(c, (double)p));
    if (threadIdx.x == 0) {
        const float2 v = ab[(int64_t)j * ld + ie];
        cetra_event ev;
        ev.depth = __ddiv_rn((double)v.x, (double)v.y);
        ev.depth_var = __ddiv_rn(1.0, (double)v.y);
        ev.dlogl = 0.5 * __dmul_rn((double)v.x, ev.depth);
        ev.t0 = __dadd_rn(t_ref, __ddiv_rn(__dmul_rn((double)(ie * p - n_pad * q), c), (double)q));
        ev.duration = durations[j];
        ev.i = ie;
        ev.j = j;
        ev.pad_ = 0;
        events[e] = ev;
        *n_events = e + 1;
    }
    const double span = ceil(h);
    const int64_t r = span < (double)I ? (int64_t)span : I;
    const int64_t lo = max((int64_t)0, ie - r), hi = min(I - 1, ie + r);
    for (int64_t i = lo + threadIdx.x; i <= hi; i += blockDim.x)
        if ((double)llabs(i - ie) < h) keys[i] = 0ull;
}

unsigned blocks_for(int64_t n, int num_sms) {
    int64_t b = (n + NB_THREADS - 1) / NB_THREADS;
    const int64_t cap = (int64_t)num_sms * 8;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

cudaError_t launch_mask(cetra_ctx *ctx, const cetra_plan *plan, float2 *grid, double P,
                        double t0, double h, unsigned long long *counts) {
    mask_kernel<<<blocks_for(plan->n_grid, ctx->num_sms), NB_THREADS, 0, ctx->stream>>>(
        grid, plan->n_grid, plan->t_ref, plan->cadence, plan->n_pad, P, t0, h, counts);
    ctx->launches++;
    return cudaGetLastError();
}

size_t mono_scratch_words(const cetra_plan *plan, int max_events) {
    return (size_t)plan->n_t0 + (size_t)max_events;
}

cudaError_t launch_monotransits(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                                unsigned long long *scratch, int max_events,
                                cetra_event *events, int *n_events) {
    const int64_t I = plan->n_t0;
    unsigned long long *keys = scratch, *slots = scratch + I;
    cudaError_t e = cudaMemsetAsync(slots, 0, (size_t)max_events * sizeof(unsigned long long),
                                    ctx->stream);
    if (!e) e = cudaMemsetAsync(n_events, 0, sizeof(int), ctx->stream);
    if (e) return e;
    const unsigned blocks = blocks_for(I, ctx->num_sms);
    mono_keys_kernel<<<blocks, NB_THREADS, 0, ctx->stream>>>(ab, plan->ab_ld, I, plan->J, keys);
    ctx->launches++;
    if ((e = cudaGetLastError())) return e;
    for (int m = 0; m < max_events; ++m) {
        mono_pick_kernel<<<blocks, NB_THREADS, 0, ctx->stream>>>(keys, I, m, slots);
        mono_event_kernel<<<1, NB_THREADS, 0, ctx->stream>>>(
            slots, m, ab, plan->ab_ld, I, plan->d_durations, plan->t_ref, plan->cadence, plan->p,
            plan->q, plan->n_pad, keys, events, n_events);
        ctx->launches += 2;
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}
