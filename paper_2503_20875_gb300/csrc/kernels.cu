// sm_103a kernels of the CETRA hot path.
//
//   resample_kernel   Sec. 2.1.1  nearest-grid-point scatter of (W y, W), W = 1/sigma^2
//   linear_kernel     Sec. 2.2    per (duration, t0): A = sum m W y, B = sum m^2 W over the
//                                 window; depth = A/B, var = 1/B, dlogl = A^2/(2B)
//   (fold.cu)         Sec. 2.3    per group of periods: sum A and B over the epoch cells of
//                                 every (duration, phase), LR = SA^2/(2 SB), in-kernel max/argmax
//   finalize_kernel   Sec. 2.3    FP64 re-sum of each period's winner: Z, var_Z, LR, t0
//   logl0_kernel      Sec. 2.2    constant-flux log-likelihood (Eq. 1 at zero depth)
//
// Why (A, B): with Delta = A/B (the inverse-variance weighted mean of y/m with
// weights m^2 W of Sec. 2.2) Eq. 2 collapses to A^2/(2B), and Eq. 4 summed over
// epochs at the common depth Z = sum A / sum B collapses to (sum A)^2/(2 sum B).
// Null grid points (W = 0) and null windows (B = 0) then drop out of every sum
// with no branch.
#include <cfloat>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace {


// --------------------------------------------------------------------------------------------
// Sec. 2.1.1: each observation goes to the nearest grid point
// k = n_pad + floor((t - t_ref) / c + 1/2) and accumulates W = 1/sigma^2 and W y.
__global__ void resample_kernel(const double *__restrict__ time, const float *__restrict__ flux,
                                const float *__restrict__ err, int64_t n, double t_ref, double c,
                                int64_t n_pad, int64_t n_grid, int flux_is_offset,
                                float2 *__restrict__ grid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double tk = time[k];
        const float fk = flux[k], ek = err[k];
        if (!(isfinite(tk) && isfinite(fk) && isfinite(ek) && ek > 0.0f)) continue;
        const double v = floor(__dadd_rn(__ddiv_rn(__dsub_rn(tk, t_ref), c), 0.5));
        // drop points outside the planned grid (a curve that does not match its plan)
        if (!(v >= -(double)n_pad) || !(v < (double)(n_grid - n_pad))) continue;
        const int64_t bin = n_pad + (int64_t)v;
        const float wk = 1.0f / (ek * ek);
        const float yk = flux_is_offset ? fk : 1.0f - fk;
        atomicAdd(&grid[bin], make_float2(wk * yk, wk));  // (W y, W), one cell
    }
}

// --------------------------------------------------------------------------------------------
// Sec. 2.2 linear search. One block per (duration j, phase class r, tile of RB*blockDim
// consecutive outputs u of that class); t0 index i = r + q u. For class r the window
// of output u is grid points a + p u + k, k < len, with template samples tab[k]
// (tables built on the host in FP64). The block stages a chunk of the table and the
// matching span of the interleaved (W y, W) grid in shared memory with 1-D bulk copies (TMA);
// each thread slides a register window over the span and accumulates RB outputs (A, B) with
// packed FP32x2 FMAs. For p > 1 the span is read as p interleaved streams (k = p k1 + k2).
// KAHAN: every term is added with Kahan compensation (CETRA_FP32_KAHAN).

// Stage cells [x0, x0 + n) of a global array whose cells [0, nvalid) hold data into
// dst[0 .. n) (cells outside [0, nvalid) read as zero). dst must sit at a byte address that is
// 8 (x0 & 1) modulo 16, so that global cell pairs map to 16-byte units. The 16-byte aligned
// interior of the valid range goes by one bulk copy that thread 0 issues on `bar` (after
// `expect` was armed with the bytes of every copy of the chunk); the block's threads store
// the at most two odd edge cells and the zero cells, which the copy never writes. Returns
// the bytes of the bulk copy; `issue` = false only computes them.
__device__ __forceinline__ uint32_t stage_cells(float2 *dst, const float2 *__restrict__ src,
                                                int64_t x0, int n, int64_t nvalid, uint64_t *bar,
                                                bool issue) {
    const int64_t lo = x0 > 0 ? x0 : 0;
    const int64_t hi = x0 + n < nvalid ? x0 + n : nvalid;
    int64_t cs = (lo + 1) & ~(int64_t)1, ce = hi & ~(int64_t)1;
    if (ce < cs) ce = cs;
    const uint32_t bytes = hi > lo ? (uint32_t)(ce - cs) * (uint32_t)sizeof(float2) : 0u;
    if (!issue) return bytes;
    if (threadIdx.x == 0 && bytes) bulk_load(dst + (cs - x0), src + cs, bytes, bar);
    // local ranges: zeros [0, v0) and [v1, n); plain copies [v0, c0) and [c1, v1)
    const int v0 = hi > lo ? (int)(lo - x0) : n, v1 = hi > lo ? (int)(hi - x0) : n;
    const int c0 = bytes ? (int)(cs - x0) : v1, c1 = bytes ? (int)(ce - x0) : v1;
    for (int k = threadIdx.x; k < v0; k += blockDim.x) dst[k] = make_float2(0.f, 0.f);
    for (int k = v1 + threadIdx.x; k < n; k += blockDim.x) dst[k] = make_float2(0.f, 0.f);
    for (int k = v0 + threadIdx.x; k < c0; k += blockDim.x) dst[k] = src[x0 + k];
    for (int k = c1 + threadIdx.x; k < v1; k += blockDim.x) dst[k] = src[x0 + k];
    return bytes;
}

// One window's outputs: (A, B) into the grid row j, and the three Sec. 2.2 outputs (depth
// A/B, its variance 1/B, ΔlogL A²/(2B)) when requested; NaN where B = 0 (a null window).
__device__ __forceinline__ void linear_store(float2 v, int64_t i, int j, int64_t I, int64_t ld,
                                             float2 *__restrict__ ab, float *__restrict__ depth,
                                             float *__restrict__ var, float *__restrict__ dlogl) {
    const int64_t idx = (int64_t)j * I + i;
    const float A = v.x, B = v.y;
    ab[(int64_t)j * ld + i] = v;
    const bool good = B > 0.0f;
    if (depth) depth[idx] = good ? A / B : __int_as_float(0x7fc00000);
    if (var) var[idx] = good ? 1.0f / B : __int_as_float(0x7fc00000);
    if (dlogl) dlogl[idx] = good ? 0.5f * (A * (A / B)) : __int_as_float(0x7fc00000);
}

template <int RB, bool KAHAN, int PFIX>
__device__ __forceinline__ void linear_block(int tile, int jr, const float2 *__restrict__ grid,
              int64_t n_grid, const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
              const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off,
              int64_t n_table, int p_arg, int q, int64_t I, int64_t ld, int kc_max,
              float2 *__restrict__ ab, float *__restrict__ depth, float *__restrict__ var,
              float *__restrict__ dlogl, int *__restrict__ status) {
    // PFIX = 1: the t0 step equals the cadence (p = 1, the common case), known at compile time
    // so that the inner loop's shared-memory offsets are immediates
    const int p = PFIX ? PFIX : p_arg;
    extern __shared__ __align__(128) float2 smem[];
    __shared__ uint64_t bar;
    const int nthr = blockDim.x;
    const int t = threadIdx.x;
    const int j = jr / q, r = jr % q;
    const int64_t U = (r < I) ? (I - r + q - 1) / q : 0;
    const int64_t UT = (int64_t)nthr * RB;
    const int64_t u0 = (int64_t)tile * UT;
    if (u0 >= U) return;  // uniform over the block
    const int padlen = win_padlen[jr];
    const int64_t a0 = (int64_t)win_a[jr] + (int64_t)p * u0;
    const int64_t toff = win_off[jr];
    // [kc_max + 2] template chunk (m, m^2), then [p UT + kc_max + 2] grid span (W y, W); each
    // shifted by one cell when its first global cell is odd (16-byte units line up)
    float2 *st_base = smem;
    float2 *sd_base = smem + ((kc_max + 3) & ~1);
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Blocked summation: `acc` collects at most LIN_SUB * RB terms before it is
    // folded into `tot`, so the FP32 rounding error grows with the block length
    // plus the number of blocks instead of with the window length.
    // With KAHAN, `tot` holds minus the compensation of `acc` instead.
    float2 acc[RB], tot[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) acc[rr] = tot[rr] = make_float2(0.f, 0.f);

    bool failed = false;
    uint32_t phase = 0;
    for (int kc0 = 0; kc0 < padlen; kc0 += kc_max) {
        const int kcl = min(kc_max, padlen - kc0);
        __syncthreads();  // the previous chunk is read
        const int64_t tx0 = toff + kc0;
        const int64_t base = a0 + kc0;
        const int dl = (int)(p * UT) + kcl;
        float2 *st = st_base + (tx0 & 1);
        float2 *sd = sd_base + (base & 1);
        if (t == 0) {
            const uint32_t bytes = stage_cells(st, tables, tx0, kcl, n_table, &bar, false) +
                                   stage_cells(sd, grid, base, dl, n_grid, &bar, false);
            fence_proxy_async();
            mbar_expect_tx(&bar, bytes);
        }
        __syncthreads();  // armed before any copy can complete
        stage_cells(st, tables, tx0, kcl, n_table, &bar, true);
        stage_cells(sd, grid, base, dl, n_grid, &bar, true);
        const bool ok = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {  // a copy did not land in time: stop (outputs NaN)
            failed = true;
            break;
        }
        const int nk1 = kcl / p;  // a multiple of RB (tables are padded to p*RB)
        for (int k2 = 0; k2 < p; ++k2) {
            const float2 *V = sd + (int64_t)p * t * RB + k2;  // V[p m]: m-th sample of stream k2
            const float2 *M = st + k2;                        // M[p k1]: template sample
            float2 buf[RB];
#pragma unroll
            for (int rr = 0; rr < RB; ++rr) buf[rr] = V[p * rr];
            for (int kb0 = 0; kb0 < nk1; kb0 += LIN_SUB * RB) {
                const int kb_end = min(nk1, kb0 + LIN_SUB * RB);
                for (int kb = kb0; kb < kb_end; kb += RB) {
#pragma unroll
                    for (int s = 0; s < RB; ++s) {
                        const int k1 = kb + s;
                        const float2 mm = M[p * k1];
#pragma unroll
                        for (int rr = 0; rr < RB; ++rr) {
                            if constexpr (KAHAN)
                                kahan_fma2(acc[rr], tot[rr], mm, buf[(s + rr) % RB]);
                            else
                                fma2(acc[rr], mm, buf[(s + rr) % RB]);
                        }
                        buf[s] = V[p * (k1 + RB)];
                    }
                }
                if constexpr (!KAHAN) {
#pragma unroll
                    for (int rr = 0; rr < RB; ++rr) {
                        add2(tot[rr], acc[rr]);
                        acc[rr] = make_float2(0.f, 0.f);
                    }
                }
            }
        }
    }
    if (failed) {
        // wait (bounded) for the copy that did not land, so that it cannot land after the
        // block exits; record the time-out; every output of the tile is NaN, written directly
        // (the staging buffer may still receive that copy)
        if (t == 0) {
            mbar_wait(&bar, phase ^ 1u);
            atomicExch(status, CETRA_ETIMEOUT);
        }
        const float nan = __int_as_float(0x7fc00000);
        for (int rr = 0; rr < RB; ++rr) {
            const int64_t u = u0 + (int64_t)t * RB + rr;
            if (u >= U) break;
            linear_store(make_float2(nan, nan), r + (int64_t)q * u, j, I, ld, ab, depth, var,
                         dlogl);
        }
        return;
    }
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        if constexpr (KAHAN)
            add2(acc[rr], tot[rr]);  // fold the last compensation in
        else
            acc[rr] = tot[rr];
    }

    // A thread holds RB consecutive t0 of the tile; a warp's direct stores would touch a
    // separate 32-byte sector per lane. The sums go through shared memory (the staged chunk
    // is no longer read) so that consecutive lanes store consecutive t0.
    __syncthreads();
    float2 *so = smem;  // UT cells: the dynamic buffer holds at least p UT + 2 kc_max + 4
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) so[t * RB + rr] = acc[rr];
    __syncthreads();
    const int nU = (int)min(UT, U - u0);
    for (int k = t; k < nU; k += nthr)
        linear_store(so[k], r + (int64_t)q * (u0 + k), j, I, ld, ab, depth, var, dlogl);
}

template <int RB, bool KAHAN>
__global__ void __launch_bounds__(128, LIN_MIN_BLOCKS)
linear_kernel(const float2 *__restrict__ grid, int64_t n_grid,
              const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
              const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off,
              int64_t n_table, int p, int q, int64_t I, int64_t ld, int kc_max,
              const int32_t *__restrict__ order, float2 *__restrict__ ab,
              float *__restrict__ depth, float *__restrict__ var, float *__restrict__ dlogl,
              int *__restrict__ status) {
    // rows by decreasing window length: blocks are dispatched in y-major order, so the
    // longest blocks start first and the last wave holds the shortest ones
    if (p == 1)
        linear_block<RB, KAHAN, 1>(blockIdx.x, order[blockIdx.y], grid, n_grid, tables, win_a,
                                   win_padlen, win_off, n_table, p, q, I, ld, kc_max, ab, depth,
                                   var, dlogl, status);
    else
        linear_block<RB, KAHAN, 0>(blockIdx.x, order[blockIdx.y], grid, n_grid, tables, win_a,
                                   win_padlen, win_off, n_table, p, q, I, ld, kc_max, ab, depth,
                                   var, dlogl, status);
}


// --------------------------------------------------------------------------------------------
// Sec. 2.3: the per-period winner, re-summed in FP64 from the FP32 grid.
__global__ void finalize_kernel(const float2 *__restrict__ ab, int64_t I, int64_t ld,
                                const double *__restrict__ durations,
                                const double *__restrict__ periods, int K,
                                const unsigned long long *__restrict__ keys,
                                const int *__restrict__ status, double t_ref, double c,
                                int64_t p, int64_t q, int64_t n_pad, double *dlogl, double *t0,
                                double *dur, double *depth, double *var, int64_t *oi, int32_t *oj) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const unsigned long long key = keys[k];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (key == 0ull || *status != 0) {  // null period, or the fold gave up
        if (dlogl) dlogl[k] = nan;
        if (t0) t0[k] = nan;
        if (dur) dur[k] = nan;
        if (depth) depth[k] = nan;
        if (var) var[k] = nan;
        if (oi) oi[k] = -1;
        if (oj) oj[k] = -1;
        return;
    }
    const uint32_t flat = 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull);
    const int64_t j = (int64_t)flat / I, i = (int64_t)flat % I;
    const double Ps = period_steps(periods[k], c, p, q);
    const float2 *row = ab + j * ld;
    double SA = 0.0, SB = 0.0;
    for (int64_t e = 0;; ++e) {
        const int64_t cell = i + epoch_offset(e, Ps);
        if (cell >= I) break;
        const float2 v = row[cell];
        SA = __dadd_rn(SA, (double)v.x);
        SB = __dadd_rn(SB, (double)v.y);
    }
    const double Z = __ddiv_rn(SA, SB);
    if (dlogl) dlogl[k] = 0.5 * __dmul_rn(SA, Z);
    if (depth) depth[k] = Z;
    if (var) var[k] = __ddiv_rn(1.0, SB);
    if (t0)
        t0[k] = __dadd_rn(t_ref, __ddiv_rn(__dmul_rn((double)(i * p - n_pad * q), c), (double)q));
    if (dur) dur[k] = durations[j];
    if (oi) oi[k] = i;
    if (oj) oj[k] = (int32_t)j;
}

// --------------------------------------------------------------------------------------------
// Sec. 2.2 (last paragraph): logL0 = sum over non-null grid points of
// -1/2 y^2 W - 1/2 ln(2 pi / W), y = (W y) / W, accumulated in FP64.
__global__ void logl0_kernel(const float2 *__restrict__ grid, int64_t n, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const float2 cell = grid[k];
        const double W = (double)cell.y;
        if (!(W > 0.0)) continue;
        const double y = (double)cell.x / W;
        acc += -0.5 * y * y * W - 0.5 * log(6.283185307179586 / W);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) atomicAdd(out, acc);
    }
}

// ============================================================================================
// Batched form: many light curves in one launch per stage.

// Index of the curve owning item x of a CSR prefix array off[0..n] (off[c] <= x < off[c+1]).

// Sec. 2.1.1 for every point of every curve (curve found from the point index).
__global__ void batch_resample_kernel(const double *__restrict__ time,
                                      const float *__restrict__ flux,
                                      const float *__restrict__ err, int64_t n,
                                      const int64_t *__restrict__ pt_off, int n_curves,
                                      const batch_curve *__restrict__ curves, double c,
                                      int64_t n_pad, int flux_is_offset,
                                      float2 *__restrict__ grid) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double tk = time[k];
        const float fk = flux[k], ek = err[k];
        if (!(isfinite(tk) && isfinite(fk) && isfinite(ek) && ek > 0.0f)) continue;
        const batch_curve cv = curves[csr_find(pt_off, n_curves, k)];
        const double v = floor(__dadd_rn(__ddiv_rn(__dsub_rn(tk, cv.t_ref), c), 0.5));
        if (!(v >= -(double)n_pad) || !(v < (double)((int64_t)cv.n_grid - n_pad))) continue;
        const int64_t bin = cv.grid_off + n_pad + (int64_t)v;
        const float wk = 1.0f / (ek * ek);
        const float yk = flux_is_offset ? fk : 1.0f - fk;
        atomicAdd(&grid[bin], make_float2(wk * yk, wk));
    }
}

// Sec. 2.2 for every curve: x-blocks enumerate the t0 tiles of all curves.
template <int RB, bool KAHAN>
__global__ void __launch_bounds__(128, LIN_MIN_BLOCKS)
batch_linear_kernel(const int64_t *__restrict__ tile_off, int n_curves,
                    const batch_curve *__restrict__ curves, const float2 *__restrict__ grid,
                    const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
                    const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off,
                    int64_t n_table, int p, int q, int kc_max, const int32_t *__restrict__ order,
                    float2 *__restrict__ ab, int *__restrict__ status) {
    const int cidx = csr_find(tile_off, n_curves, blockIdx.x);
    const batch_curve cv = curves[cidx];
    if (cv.I <= 0) return;
    if (p == 1)
        linear_block<RB, KAHAN, 1>((int)(blockIdx.x - tile_off[cidx]), order[blockIdx.y],
                                   grid + cv.grid_off, cv.n_grid, tables, win_a, win_padlen,
                                   win_off, n_table, p, q, cv.I, cv.ld, kc_max, ab + cv.ab_off,
                                   nullptr, nullptr, nullptr, status);
    else
        linear_block<RB, KAHAN, 0>((int)(blockIdx.x - tile_off[cidx]), order[blockIdx.y],
                                   grid + cv.grid_off, cv.n_grid, tables, win_a, win_padlen,
                                   win_off, n_table, p, q, cv.I, cv.ld, kc_max, ab + cv.ab_off,
                                   nullptr, nullptr, nullptr, status);
}

// The winner of every curve: its best period from the curve key, that period's best
// (duration, t0) from its own key, re-summed in FP64.
__global__ void batch_finalize_kernel(const float2 *__restrict__ ab,
                                      const batch_curve *__restrict__ curves, int n_curves,
                                      const double *__restrict__ durations, double c, int64_t p,
                                      int64_t q, int64_t n_pad,
                                      const unsigned long long *__restrict__ period_keys,
                                      const unsigned long long *__restrict__ curve_keys,
                                      const int *__restrict__ status,
                                      cetra_best *__restrict__ best) {
    const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= n_curves) return;
    const batch_curve cv = curves[cidx];
    const unsigned long long key = curve_keys[cidx];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    cetra_best out;
    out.dlogl = out.period = out.t0 = out.duration = out.depth = out.depth_var = nan;
    out.k = out.i = -1;
    out.j = -1;
    out.n_periods = cv.n_periods;
    if (key == 0ull || *status != 0) {
        best[cidx] = out;
        return;
    }
    const int64_t k = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
    const unsigned long long pk = period_keys[cv.per_off + k];
    const uint32_t flat = 0xFFFFFFFFu - (uint32_t)(pk & 0xFFFFFFFFull);
    const int j = (int)(flat / (uint32_t)cv.I), i = (int)(flat % (uint32_t)cv.I);
    const double P = batch_period(cv.pmin, cv.ratio, k);
    const double Ps = period_steps(P, c, p, q);
    const float2 *row = ab + cv.ab_off + (int64_t)j * cv.ld;
    double SA = 0.0, SB = 0.0;
    for (int64_t e = 0;; ++e) {
        const int64_t cell = i + epoch_offset(e, Ps);
        if (cell >= cv.I) break;
        SA = __dadd_rn(SA, (double)row[cell].x);
        SB = __dadd_rn(SB, (double)row[cell].y);
    }
    const double Z = __ddiv_rn(SA, SB);
    out.dlogl = 0.5 * __dmul_rn(SA, Z);
    out.period = P;
    out.t0 = __dadd_rn(cv.t_ref, __ddiv_rn(__dmul_rn((double)((int64_t)i * p - n_pad * q), c),
                                          (double)q));
    out.duration = durations[j];
    out.depth = Z;
    out.depth_var = __ddiv_rn(1.0, SB);
    out.k = k;
    out.i = i;
    out.j = j;
    best[cidx] = out;
}

// Learned-proposal selection (not in the paper), one block per curve. Interval q < n_int
// spans [e_q, e_{q+1}) days with e_q = p_lo (p_hi / p_lo)^(q / n_int); kst[q] = the number of
// the curve's periods below e_q (so interval q holds periods kst[q] .. kst[q+1] - 1). Of the
// intervals holding at least one period ("present"), the max(1, ceil(top_frac n_present))
// with the highest scores are kept (NaN ranks lowest; ties: lower q first), and every
// 8-period group holding a period of a kept interval becomes one fold work item. Items are
// appended to items[] behind the counter counts[0] (their order across curves is not fixed);
// counts[1] accumulates the periods of the selected groups. flags: one byte per work item of
// the batch (scratch).
constexpr int SEL_THREADS = 256;
__global__ void __launch_bounds__(SEL_THREADS)
batch_select_kernel(const batch_curve *__restrict__ curves, const int64_t *__restrict__ group_off,
                    const float *__restrict__ scores, int n_int, double p_lo, double p_hi,
                    double top_frac, unsigned char *__restrict__ flags,
                    int64_t *__restrict__ items, unsigned long long *__restrict__ counts) {
    __shared__ int64_t kst[SEL_MAX_INTERVALS + 1];
    __shared__ float sc[SEL_MAX_INTERVALS];
    __shared__ unsigned char keep[SEL_MAX_INTERVALS];
    __shared__ int s_present;
    __shared__ unsigned long long s_base;
    __shared__ int s_warp[SEL_THREADS / 32];
    __shared__ unsigned long long s_per[SEL_THREADS / 32];
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const batch_curve cv = curves[c];
    const int64_t K = cv.n_periods;
    if (K <= 0) return;  // uniform over the block
    const double lr = log(cv.ratio);
    for (int q = tid; q <= n_int; q += SEL_THREADS) {
        const double edge = p_lo * pow(p_hi / p_lo, (double)q / n_int);
        const double est = ceil(log(edge / cv.pmin) / lr);
        int64_t k = !(est > 0.0) ? 0 : (est >= (double)K ? K : (int64_t)est);
        while (k > 0 && batch_period(cv.pmin, cv.ratio, k - 1) >= edge) --k;
        while (k < K && batch_period(cv.pmin, cv.ratio, k) < edge) ++k;
        kst[q] = k;
    }
    if (tid == 0) s_present = 0;
    __syncthreads();
    int mine = 0;
    for (int q = tid; q < n_int; q += SEL_THREADS) {
        const float v = scores[(int64_t)c * n_int + q];
        sc[q] = v == v ? v : -INFINITY;
        mine += kst[q + 1] > kst[q];
    }
    atomicAdd(&s_present, mine);
    __syncthreads();
    const int n_present = s_present;
    if (n_present == 0) return;  // uniform
    const int n_keep = max(1, (int)ceil(top_frac * (double)n_present));
    for (int q = tid; q < n_int; q += SEL_THREADS) {
        unsigned char k = 0;
        if (kst[q + 1] > kst[q]) {
            const float v = sc[q];
            int rank = 0;
            for (int r = 0; r < n_int; ++r)
                rank += (kst[r + 1] > kst[r]) && (sc[r] > v || (sc[r] == v && r < q));
            k = rank < n_keep;
        }
        keep[q] = k;
    }
    const int64_t g0 = group_off[c], G = (K + FT_G - 1) / FT_G;
    for (int64_t g = tid; g < G; g += SEL_THREADS) flags[g0 + g] = 0;
    __syncthreads();
    for (int q = 0; q < n_int; ++q) {
        if (!keep[q]) continue;  // uniform: keep[] is shared
        const int64_t lo = kst[q] / FT_G, hi = (kst[q + 1] - 1) / FT_G;
        for (int64_t g = lo + tid; g <= hi; g += SEL_THREADS) flags[g0 + g] = 1;
    }
    __syncthreads();
    for (int64_t base = 0; base < G; base += SEL_THREADS) {
        const int64_t g = base + tid;
        const bool f = g < G && flags[g0 + g];
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        unsigned long long per = f ? (unsigned long long)min((int64_t)FT_G, K - g * FT_G) : 0ull;
        for (int o = 16; o > 0; o >>= 1) per += __shfl_down_sync(0xFFFFFFFFu, per, o);
        if (lane == 0) {
            s_warp[wid] = __popc(bal);
            s_per[wid] = per;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long tot = 0, ptot = 0;
            for (int w = 0; w < SEL_THREADS / 32; ++w) {
                const int n = s_warp[w];
                s_warp[w] = (int)tot;  // exclusive prefix over warps
                tot += n;
                ptot += s_per[w];
            }
            s_base = tot ? atomicAdd(&counts[0], tot) : 0ull;
            if (ptot) atomicAdd(&counts[1], ptot);
        }
        __syncthreads();
        if (f) items[s_base + s_warp[wid] + __popc(bal & ((1u << lane) - 1u))] = g0 + g;
        __syncthreads();
    }
}

// Linear-search features of every batch curve: the window LR = A^2 / (2B) (Sec. 2.2) of
// the windows with a positive depth (A > 0: a dimming), max-pooled over n_bins equal bins
// of the curve's t0 grid (bin width ceil(I / n_bins)); empty bins, null windows and
// brightenings give 0. Layout [curve][duration][bin].
__global__ void batch_features_kernel(const float2 *__restrict__ ab,
                                      const batch_curve *__restrict__ curves, int n_curves, int J,
                                      int n_bins, float *__restrict__ out) {
    const int64_t total = (int64_t)n_curves * J * n_bins;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        const int bin = (int)(x % n_bins);
        const int j = (int)((x / n_bins) % J);
        const int cidx = (int)(x / ((int64_t)n_bins * J));
        const batch_curve cv = curves[cidx];
        float m = 0.0f;
        if (cv.I > 0) {
            const int width = (cv.I + n_bins - 1) / n_bins;
            const int lo = bin * width, hi = min(cv.I, lo + width);
            const float2 *row = ab + cv.ab_off + (int64_t)j * cv.ld;
            for (int i = lo; i < hi; ++i) {
                const float2 v = row[i];
                if (v.y > 0.0f && v.x > 0.0f) m = fmaxf(m, 0.5f * (v.x * (v.x / v.y)));
            }
        }
        out[x] = m;
    }
}

// Self-test of the bounded barrier wait every fold uses: a barrier expects bytes that no copy
// will deliver, so its phase never completes; the wait must give up after FT_WAIT_CYCLES and
// report it (out[0] = 1), and the kernel must return normally.
// --------------------------------------------------------------------------------------------
// Measured ceilings of the two stages' bounds. The linear search is bound by packed FP32 FMA
// issue, the fold by 8-byte shared-memory loads each added into a packed FP32 sum; these
// kernels run each pattern alone, at full occupancy, with PEAK_CHAINS independent chains a
// thread (enough to cover the pipe latencies), and store their sums so nothing is dead code.
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_SMEM_CELLS = 2 * PEAK_CHAINS * PEAK_THREADS;  // float2 per block (32 KiB)

__global__ void __launch_bounds__(PEAK_THREADS) peak_fma_kernel(float2 a, float2 b, int iters,
                                                                float *__restrict__ out) {
    float2 acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = make_float2((float)threadIdx.x, (float)k);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) fma2(acc[k], a, b);
    float r = 0.0f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) r += acc[k].x + acc[k].y;
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// A volatile load: the buffer is never written in the loop, and a plain load could be lifted
// out of it, leaving only the adds to time.
__device__ __forceinline__ float2 lds2(uint32_t addr) {
    float2 v;
    asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// Thread t reads cells t + PEAK_THREADS k (+ half the buffer on odd iterations): every warp
// load is 256 contiguous bytes, conflict-free, as in the fold.
__global__ void __launch_bounds__(PEAK_THREADS) peak_smem_kernel(int iters,
                                                                 float *__restrict__ out) {
    __shared__ float2 s[PEAK_SMEM_CELLS];
    for (int x = threadIdx.x; x < PEAK_SMEM_CELLS; x += blockDim.x)
        s[x] = make_float2((float)x, 1.0f);
    __syncthreads();
    float2 acc[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) acc[k] = make_float2(0.0f, 0.0f);
    const uint32_t base = smem_u32(s + threadIdx.x);
    constexpr uint32_t half = PEAK_SMEM_CELLS / 2 * sizeof(float2);
    for (int it = 0; it < iters; ++it) {
        const uint32_t p = base + ((uint32_t)it & 1u) * half;
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k)
            add2(acc[k], lds2(p + (uint32_t)(k * PEAK_THREADS * sizeof(float2))));
    }
    float r = 0.0f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) r += acc[k].x + acc[k].y;
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void wait_timeout_selftest_kernel(int *out, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, 16);  // arrives and expects 16 bytes that never come
        const long long t0 = clock64();
        const bool ok = mbar_wait(&bar, 0);
        // a wait that gave up is recorded the way the fold records it
        if (!ok && status) atomicExch(status, CETRA_ETIMEOUT);
        if (out) {
            out[0] = ok ? 0 : 1;
            out[1] = (int)min((clock64() - t0) >> 20, (long long)INT32_MAX);  // ~2^20-cycle units
        }
    }
}

}  // namespace

// ============================================================================================
// launchers

cudaError_t launch_resample(cetra_ctx *ctx, const cetra_plan *plan, const double *time,
                            const float *flux, const float *err, int64_t n, float2 *grid) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    blocks = blocks > (int64_t)ctx->num_sms * 16 ? (int64_t)ctx->num_sms * 16 : blocks;
    prof_mark(ctx, KID_RESAMPLE, true);
    resample_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(
        time, flux, err, n, plan->t_ref, plan->cadence, plan->n_pad, plan->n_grid,
        plan->flux_is_offset, grid);
    prof_mark(ctx, KID_RESAMPLE, false);
    ctx->launches++;
    return cudaGetLastError();
}

#ifndef LIN_THREADS
#define LIN_THREADS 128  // threads per linear block (RB outputs each)
#endif
#ifndef LIN_KC
#define LIN_KC 2304      // template samples per staged table chunk (before rounding to p RB)
#endif

cudaError_t linear_configure(cetra_plan *plan, const cetra_ctx *ctx) {
    const int p = (int)plan->p;
    const size_t budget = 100 * 1024;  // keeps two blocks resident per SM at the largest shape
    const int unit = p * LIN_RB;
    int kc = (LIN_KC / unit) * unit;
    if (kc < unit) kc = unit;
    if (plan->max_padlen > 0 && kc > plan->max_padlen) kc = plan->max_padlen;
    int threads = LIN_THREADS;
    auto bytes = [&](int th, int k) { return linear_smem_bytes(p, th, k); };
    while (threads > 32 && bytes(threads, kc) > budget) threads /= 2;
    while (kc > unit && bytes(threads, kc) > budget) kc -= unit;
    plan->lin_threads = threads;
    plan->lin_kc = kc;
    plan->lin_smem = bytes(threads, kc);
    size_t limit = ctx->max_smem_optin ? ctx->max_smem_optin : 227 * 1024;
    if (plan->lin_smem > limit) return cudaErrorInvalidConfiguration;
    for (auto fn : {linear_kernel<LIN_RB, false>, linear_kernel<LIN_RB, true>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan->lin_smem);
        if (e != cudaSuccess) return e;
    }
    return fold_configure();
}

cudaError_t launch_linear(cetra_ctx *ctx, const cetra_plan *plan, const float2 *grid, float2 *ab,
                          float *depth, float *var, float *dlogl, int *status) {
    const int64_t I = plan->n_t0, q = plan->q;
    const int64_t Umax = (I + q - 1) / q;
    const int64_t UT = (int64_t)plan->lin_threads * LIN_RB;
    const int64_t gx = (Umax + UT - 1) / UT;
    if (gx == 0) return cudaSuccess;
    dim3 blocks((unsigned)gx, (unsigned)(plan->J * q));
    prof_mark(ctx, KID_LINEAR, true);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? linear_kernel<LIN_RB, true>
                                                    : linear_kernel<LIN_RB, false>;
    kern<<<blocks, plan->lin_threads, plan->lin_smem, ctx->stream>>>(
        grid, plan->n_grid, plan->d_tables, plan->d_win_a, plan->d_win_padlen, plan->d_win_off,
        (int64_t)plan->tables.size(), (int)plan->p, (int)q, I, plan->ab_ld, plan->lin_kc,
        plan->d_lin_order, ab, depth, var, dlogl, status);
    prof_mark(ctx, KID_LINEAR, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_finalize(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                            const double *periods, int K, const unsigned long long *keys,
                            const int *status, double *dlogl, double *t0, double *dur, double *depth, double *var,
                            int64_t *oi, int32_t *oj) {
    if (K <= 0) return cudaSuccess;
    const int threads = 128;
    prof_mark(ctx, KID_FINALIZE, true);
    finalize_kernel<<<(K + threads - 1) / threads, threads, 0, ctx->stream>>>(
        ab, plan->n_t0, plan->ab_ld, plan->d_durations, periods, K, keys, status, plan->t_ref,
        plan->cadence, plan->p,
        plan->q, plan->n_pad, dlogl, t0, dur, depth, var, oi, oj);
    prof_mark(ctx, KID_FINALIZE, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_logl0(cetra_ctx *ctx, const cetra_plan *plan, const float2 *grid,
                         double *out) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), ctx->stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    int64_t blocks = (plan->n_grid + threads - 1) / threads;
    if (blocks > (int64_t)ctx->num_sms * 4) blocks = (int64_t)ctx->num_sms * 4;
    if (blocks < 1) blocks = 1;
    prof_mark(ctx, KID_LOGL0, true);
    logl0_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(grid, plan->n_grid, out);
    prof_mark(ctx, KID_LOGL0, false);
    ctx->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- batched

double batch_period_host(double pmin, double ratio, int64_t k) {
    double x = 1.0, b = ratio;
    while (k) {
        if (k & 1) x = x * b;
        b = b * b;
        k >>= 1;
    }
    return pmin * x;
}

cudaError_t launch_batch_resample(cudaStream_t stream, int num_sms, const cetra_plan *plan,
                                  const double *time, const float *flux, const float *err,
                                  int64_t n_points, const int64_t *pt_offsets, int n_curves,
                                  const batch_curve *curves, float2 *grid) {
    if (n_points <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n_points + threads - 1) / threads;
    if (blocks > (int64_t)num_sms * 32) blocks = (int64_t)num_sms * 32;
    batch_resample_kernel<<<(unsigned)blocks, threads, 0, stream>>>(
        time, flux, err, n_points, pt_offsets, n_curves, curves, plan->cadence, plan->n_pad,
        plan->flux_is_offset, grid);
    return cudaGetLastError();
}

cudaError_t launch_batch_linear(cudaStream_t stream, const cetra_plan *plan, int threads,
                                const int64_t *tile_off, int n_curves, int64_t n_tiles,
                                const batch_curve *curves, const float2 *grid, float2 *ab,
                                int *status) {
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 2147483647) return cudaErrorInvalidConfiguration;
    dim3 blocks((unsigned)n_tiles, (unsigned)(plan->J * plan->q));
    const size_t smem = linear_smem_bytes((int)plan->p, threads, plan->lin_kc);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? batch_linear_kernel<LIN_RB, true>
                                                    : batch_linear_kernel<LIN_RB, false>;
    kern<<<blocks, threads, smem, stream>>>(tile_off, n_curves, curves, grid, plan->d_tables,
                                            plan->d_win_a, plan->d_win_padlen, plan->d_win_off,
                                            (int64_t)plan->tables.size(), (int)plan->p,
                                            (int)plan->q, plan->lin_kc, plan->d_lin_order, ab,
                                            status);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(cudaStream_t stream, const cetra_plan *plan, const float2 *ab,
                                  const batch_curve *curves, int n_curves,
                                  const unsigned long long *period_keys,
                                  const unsigned long long *curve_keys, const int *status,
                                  cetra_best *best) {
    if (n_curves <= 0) return cudaSuccess;
    const int threads = 128;
    batch_finalize_kernel<<<(n_curves + threads - 1) / threads, threads, 0, stream>>>(
        ab, curves, n_curves, plan->d_durations, plan->cadence, plan->p, plan->q, plan->n_pad,
        period_keys, curve_keys, status, best);
    return cudaGetLastError();
}

cudaError_t launch_batch_select(cudaStream_t stream, const batch_curve *curves,
                                const int64_t *group_off, int n_curves, const float *scores,
                                int n_int, double p_lo, double p_hi, double top_frac,
                                unsigned char *flags, int64_t *items,
                                unsigned long long *counts) {
    if (n_curves <= 0) return cudaSuccess;
    batch_select_kernel<<<n_curves, SEL_THREADS, 0, stream>>>(curves, group_off, scores, n_int,
                                                              p_lo, p_hi, top_frac, flags, items,
                                                              counts);
    return cudaGetLastError();
}

cudaError_t batch_configure(const cetra_plan *plan) {
    const size_t lin_max = linear_smem_bytes((int)plan->p, 128, plan->lin_kc);
    for (auto fn : {batch_linear_kernel<LIN_RB, false>, batch_linear_kernel<LIN_RB, true>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)lin_max);
        if (e != cudaSuccess) return e;
    }
    return fold_configure();
}

cudaError_t launch_batch_features(cudaStream_t stream, int num_sms, const cetra_plan *plan,
                                  const float2 *ab, const batch_curve *curves, int n_curves,
                                  int n_bins, float *out) {
    const int64_t total = (int64_t)n_curves * plan->J * n_bins;
    if (total <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > (int64_t)num_sms * 32) blocks = (int64_t)num_sms * 32;
    batch_features_kernel<<<(unsigned)blocks, threads, 0, stream>>>(ab, curves, n_curves, plan->J,
                                                                     n_bins, out);
    return cudaGetLastError();
}

cudaError_t launch_wait_timeout_selftest(cudaStream_t stream, int *d_out, int *d_status) {
    wait_timeout_selftest_kernel<<<1, 32, 0, stream>>>(d_out, d_status);
    return cudaGetLastError();
}

int peak_grid(int num_sms, bool smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, smem ? (const void *)peak_smem_kernel : (const void *)peak_fma_kernel,
            PEAK_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return num_sms * per_sm;
}

cudaError_t launch_peak(cudaStream_t stream, bool smem, int blocks, int iters, float *d_out,
                        double *work) {
    const double lanes = (double)blocks * PEAK_THREADS * iters * PEAK_CHAINS;
    if (smem) {
        peak_smem_kernel<<<blocks, PEAK_THREADS, 0, stream>>>(iters, d_out);
        *work = lanes * sizeof(float2);  // bytes loaded
    } else {
        peak_fma_kernel<<<blocks, PEAK_THREADS, 0, stream>>>(make_float2(1e-3f, 2e-3f),
                                                             make_float2(1e-3f, 5e-4f), iters,
                                                             d_out);
        *work = lanes * 4.0;  // two FMA lanes, 2 flop each
    }
    return cudaGetLastError();
}
