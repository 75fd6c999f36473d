// sm_103a kernels of the CETRA hot path.
//
//   resample_kernel   Sec. 2.1.1  nearest-grid-point scatter of (W y, W), W = 1/sigma^2
//   linear_kernel     Sec. 2.2    per (duration, t0): A = sum m W y, B = sum m^2 W over the
//                                 window; depth = A/B, var = 1/B, dlogl = A^2/(2B)
//   fold_tma_kernel   Sec. 2.3    per group of periods: sum A and B over the epoch cells of
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

#include "internal.h"

namespace {

__device__ __forceinline__ unsigned long long pack2(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

// acc += a * b elementwise with one packed FP32x2 fused multiply-add.
__device__ __forceinline__ void fma2(float2 &acc, float2 a, float2 b) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(acc)));
    acc = unpack2(d);
}

// acc += v elementwise with one packed FP32x2 add.
__device__ __forceinline__ void add2(float2 &acc, float2 v) {
#ifdef CETRA_SCALAR_ADD
    acc.x += v.x;
    acc.y += v.y;
#else
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(acc)), "l"(pack2(v)));
    acc = unpack2(d);
#endif
}

// d = a - b elementwise with one packed FP32x2 subtract.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(d);
}

// Kahan-compensated s += a * b on (A, B) pairs; nc carries minus the running
// compensation: y = a b + nc, t = s + y, nc = y - (t - s), s = t.
__device__ __forceinline__ void kahan_fma2(float2 &s, float2 &nc, float2 a, float2 b) {
    float2 y = nc;
    fma2(y, a, b);
    float2 t = s;
    add2(t, y);
    nc = sub2(y, sub2(t, s));
    s = t;
}

// Kahan-compensated s += v on (A, B) pairs (nc as above).
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &nc, float2 v) {
    float2 y = v;
    add2(y, nc);
    float2 t = s;
    add2(t, y);
    nc = sub2(y, sub2(t, s));
    s = t;
}

// Nearest epoch cell offset o_e = floor(e Ps + 1/2), FP64, no contraction.
__device__ __forceinline__ int64_t epoch_offset(int64_t e, double Ps) {
    return (int64_t)floor(__dadd_rn(__dmul_rn((double)e, Ps), 0.5));
}

// Period in t0 steps, Ps = (P q) / (c p), FP64, no contraction.
__device__ __forceinline__ double period_steps(double P, double c, int64_t p, int64_t q) {
    return __ddiv_rn(__dmul_rn(P, (double)q), __dmul_rn(c, (double)p));
}

// --------------------------------------------------------------------------------------------
// Sec. 2.1.1: each observation goes to the nearest grid point
// k = n_pad + floor((t - t_ref) / c + 1/2) and accumulates W = 1/sigma^2 and W y.
__global__ void resample_kernel(const double *__restrict__ time, const float *__restrict__ flux,
                                const float *__restrict__ err, int64_t n, double t_ref, double c,
                                int64_t n_pad, int64_t n_grid, int flux_is_offset,
                                float *__restrict__ wy, float *__restrict__ w) {
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
        atomicAdd(&wy[bin], wk * yk);
        atomicAdd(&w[bin], wk);
    }
}

// --------------------------------------------------------------------------------------------
// Sec. 2.2 linear search. One block per (duration j, phase class r, tile of RB*blockDim
// consecutive outputs u of that class); t0 index i = r + q u. For class r the window
// of output u is grid points a + p u + k, k < len, with template samples tab[k]
// (tables built on the host in FP64). The block stages a chunk of the table and the
// matching span of the (W y, W) grid in shared memory; each thread slides a register
// window over the span and accumulates RB outputs (A, B) with packed FP32x2 FMAs.
// For p > 1 the span is read as p interleaved streams (k = p k1 + k2).
// KAHAN: every term is added with Kahan compensation (CETRA_FP32_KAHAN).
constexpr int LIN_STAGE_U = 4;  // staging loads in flight per thread (linear kernel)
template <int RB, bool KAHAN, int PFIX>
__device__ __forceinline__ void linear_block(int tile, int jr, const float *__restrict__ wy,
              const float *__restrict__ w, int64_t n_grid,
              const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
              const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off,
              int p_arg, int q, int64_t I, int64_t ld, int kc_max, float2 *__restrict__ ab,
              float *__restrict__ depth,
              float *__restrict__ var, float *__restrict__ dlogl) {
    // PFIX = 1: the t0 step equals the cadence (p = 1, the common case), known at compile time
    // so that the inner loop's shared-memory offsets are immediates
    const int p = PFIX ? PFIX : p_arg;
    extern __shared__ float2 smem[];
    const int nthr = blockDim.x;
    const int t = threadIdx.x;
    const int j = jr / q, r = jr % q;
    const int64_t U = (r < I) ? (I - r + q - 1) / q : 0;
    const int64_t UT = (int64_t)nthr * RB;
    const int64_t u0 = (int64_t)tile * UT;
    if (u0 >= U) return;
    const int padlen = win_padlen[jr];
    const int64_t a0 = (int64_t)win_a[jr] + (int64_t)p * u0;
    const float2 *tab = tables + win_off[jr];
    float2 *st = smem;           // [kc_max] template chunk (m, m^2)
    float2 *sd = smem + kc_max;  // [p*UT + kc_max] grid span (W y, W)

    // Blocked summation: `acc` collects at most LIN_SUB * RB terms before it is
    // folded into `tot`, so the FP32 rounding error grows with the block length
    // plus the number of blocks instead of with the window length.
    // With KAHAN, `tot` holds minus the compensation of `acc` instead.
    float2 acc[RB], tot[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) acc[rr] = tot[rr] = make_float2(0.f, 0.f);

    for (int kc0 = 0; kc0 < padlen; kc0 += kc_max) {
        const int kcl = min(kc_max, padlen - kc0);
        __syncthreads();
        // staging: LIN_STAGE_U cells per thread in flight before the shared stores
        for (int idx0 = t; idx0 < kcl; idx0 += LIN_STAGE_U * nthr) {
            float2 v[LIN_STAGE_U];
#pragma unroll
            for (int u = 0; u < LIN_STAGE_U; ++u) {
                const int idx = idx0 + u * nthr;
                v[u] = idx < kcl ? tab[kc0 + idx] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < LIN_STAGE_U; ++u)
                if (idx0 + u * nthr < kcl) st[idx0 + u * nthr] = v[u];
        }
        const int64_t base = a0 + kc0;
        const int dl = (int)(p * UT) + kcl;
        for (int idx0 = t; idx0 < dl; idx0 += LIN_STAGE_U * nthr) {
            float2 v[LIN_STAGE_U];
#pragma unroll
            for (int u = 0; u < LIN_STAGE_U; ++u) {
                const int64_t n = base + idx0 + u * nthr;
                v[u] = make_float2(0.f, 0.f);
                if (idx0 + u * nthr < dl && n >= 0 && n < n_grid) v[u] = make_float2(wy[n], w[n]);
            }
#pragma unroll
            for (int u = 0; u < LIN_STAGE_U; ++u)
                if (idx0 + u * nthr < dl) sd[idx0 + u * nthr] = v[u];
        }
        __syncthreads();
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
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        if constexpr (KAHAN)
            add2(acc[rr], tot[rr]);  // fold the last compensation in
        else
            acc[rr] = tot[rr];
    }

#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int64_t u = u0 + (int64_t)t * RB + rr;
        if (u >= U) break;
        const int64_t i = r + (int64_t)q * u;
        const int64_t idx = (int64_t)j * I + i;
        const float A = acc[rr].x, B = acc[rr].y;
        ab[(int64_t)j * ld + i] = acc[rr];
        const bool ok = B > 0.0f;
        if (depth) depth[idx] = ok ? A / B : __int_as_float(0x7fc00000);
        if (var) var[idx] = ok ? 1.0f / B : __int_as_float(0x7fc00000);
        if (dlogl) dlogl[idx] = ok ? 0.5f * (A * (A / B)) : __int_as_float(0x7fc00000);
    }
}

template <int RB, bool KAHAN>
__global__ void __launch_bounds__(128, 4)
linear_kernel(const float *__restrict__ wy, const float *__restrict__ w, int64_t n_grid,
              const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
              const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off, int p,
              int q, int64_t I, int64_t ld, int kc_max, const int32_t *__restrict__ order,
              float2 *__restrict__ ab, float *__restrict__ depth, float *__restrict__ var,
              float *__restrict__ dlogl) {
    // rows by decreasing window length: blocks are dispatched in y-major order, so the
    // longest blocks start first and the last wave holds the shortest ones
    if (p == 1)
        linear_block<RB, KAHAN, 1>(blockIdx.x, order[blockIdx.y], wy, w, n_grid, tables, win_a,
                                   win_padlen, win_off, p, q, I, ld, kc_max, ab, depth, var,
                                   dlogl);
    else
        linear_block<RB, KAHAN, 0>(blockIdx.x, order[blockIdx.y], wy, w, n_grid, tables, win_a,
                                   win_padlen, win_off, p, q, I, ld, kc_max, ab, depth, var,
                                   dlogl);
}

// Per-period key: larger LR wins; on equal LR the smaller flat index j*I + i wins
// (smallest duration, then smallest t0). LR >= 0, so its float bits order like uint.
__device__ __forceinline__ unsigned long long make_key(float lr, uint32_t flat) {
    return ((unsigned long long)__float_as_uint(lr) << 32) | (unsigned long long)(0xFFFFFFFFu - flat);
}

__device__ __forceinline__ unsigned long long block_max_key(unsigned long long v,
                                                            unsigned long long *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_down_sync(0xFFFFFFFFu, v, o);
        v = u > v ? u : v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? red[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long u = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = u > v ? u : v;
        }
    }
    return v;
}

// --------------------------------------------------------------------------------------------
// Shared-memory barriers and 1-D bulk copies (TMA) used by the fold.
__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy; src and dst 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Potentially blocking test of a barrier phase: the thread may be suspended (up
// to the hinted time) instead of spinning, so waiting warps do not take issue slots.
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(FT_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within FT_WAIT_CYCLES SM clocks.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (clock64() - t0 > FT_WAIT_CYCLES) return false;
    }
}

// --------------------------------------------------------------------------------------------
// Sec. 2.3 periodic search. One block folds a group of FT_G consecutive trial periods
// over every duration. Neighbouring periods gather nearly the same epoch cells, so
// for a tile of FT_T phases and an epoch e the block copies the union of the cells
// the group needs, [i0 + min_g o_e(g), i0 + max_g o_e(g) + FT_T), into shared memory
// with one bulk copy (FT_NSTAGE-deep ring, one mbarrier per stage) and every period
// reads its cells from there: the grid is read from L2 about once per group instead
// of once per period. Thread t owns phases i0 + t + r * FT_THREADS (r < FT_R) of
// every period of the group, summing (A, B) over epochs in ascending order.
// Grid rows carry FOLD_PAD zero cells after the last t0, so a strip never needs
// clipping: cells past the end contribute (0, 0).
// Groups whose offsets spread too far apart for one strip are split (8 -> 4 -> 2 -> 1);
// a period with more epochs than the offset table holds is folded straight from
// global memory with its offsets computed in FP64 on the fly.
constexpr int32_t FT_SENT = INT32_MAX;  // epoch past the end of the t0 grid

// Shared state of the fold block.
struct fold_smem {
    uint64_t bar[FT_NSTAGE];  // stage filled (bulk copy landed)
    unsigned long long red[FT_THREADS / 32];
    unsigned long long best[FT_G][FT_THREADS];
    double P[FT_G], Ps[FT_G];
    int nph[FT_G];
    int E[FT_G];
    int bad;
    int tight;  // some epoch's spread leaves less than the sliced path's margin
};

// Ring of bulk copies: `n` counts copies issued (thread 0) or consumed (all threads);
// copy n lands in stage n % FT_NSTAGE, completing phase n / FT_NSTAGE of that stage's `bar`.
// The block meets at a barrier after every epoch (which also votes on wait time-outs), so
// thread 0 may refill the stage read two epochs earlier. (Per-stage drain barriers instead,
// with warps drifting up to two epochs apart, measured 0.6-2 % faster on the largest
// workloads but 11-13 % slower on small ones and on the compensated path.)
struct ring {
    uint32_t n = 0, stage = 0, parity = 0;
    __device__ void next() {
        ++n;
        if (++stage == FT_NSTAGE) {
            stage = 0;
            parity ^= 1u;
        }
    }
};

// The GS strip offsets of one epoch, with 16-byte shared loads where the row allows.
template <int GS>
__device__ __forceinline__ void load_offsets(const int32_t *de, int32_t *dv) {
    if constexpr (GS % 4 == 0) {
#pragma unroll
        for (int v = 0; v < GS / 4; ++v) {
            const int4 x = reinterpret_cast<const int4 *>(de)[v];
            dv[4 * v] = x.x;
            dv[4 * v + 1] = x.y;
            dv[4 * v + 2] = x.z;
            dv[4 * v + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) dv[gg] = de[gg];
    }
}

// Fold one sub-group of GS periods [g0, g0 + GS) whose table is built: offsets relative
// to the epoch's strip start, d[e][gg] = o_e(g) - tmin[e] (FT_SENT: no cell),
// tmin[e], tlen[e] (strip spread) and full[e] (every period has a cell at epoch e).
// R phases per thread (tile FT_THREADS * R <= FT_T); KAHAN: compensated epoch sums.
// Returns false if a bulk copy timed out (the block must stop).
template <int GS, int R, bool KAHAN>
__device__ bool fold_subgroup(fold_smem &sm, float2 *strips, const int32_t *tab, int Es, int g0,
                              int k0, const float2 *__restrict__ ab, int I, int64_t ld, int J,
                              const double *__restrict__ durations,
                              const uint8_t *__restrict__ mask, ring &iss, ring &con,
                              int *__restrict__ status) {
    const int t = threadIdx.x;
    const int32_t *d = tab;
    const int32_t *tmin = tab + Es * GS;
    const int32_t *tlen = tmin + Es;
    const int32_t *full = tlen + Es;
    int nph_sub = 0;
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) nph_sub = max(nph_sub, sm.nph[g0 + gg]);
    float best_lr[GS];
    uint32_t best_at[GS];
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        best_lr[gg] = -1.0f;
        best_at[gg] = 0u;
    }
    for (int j = 0; j < J && nph_sub > 0; ++j) {
        const double D = durations[j];
        unsigned use = 0u;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            const int g = g0 + gg;
            if (sm.E[g] > 0 && D < sm.P[g] && (!mask || mask[(int64_t)(k0 + g) * J + j]))
                use |= 1u << gg;
        }
        if (!use) continue;
        const bool all_used = use == (1u << GS) - 1u;
        const float2 *row = ab + (int64_t)j * ld;
        constexpr int T = FT_THREADS * R;
        for (int i0 = 0; i0 < nph_sub; i0 += T) {
            float2 acc[GS][R];
            float2 cmp[KAHAN ? GS : 1][KAHAN ? R : 1];  // minus the Kahan compensation
#pragma unroll
            for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[gg][r] = make_float2(0.f, 0.f);
            if constexpr (KAHAN) {
#pragma unroll
                for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                    for (int r = 0; r < R; ++r) cmp[gg][r] = make_float2(0.f, 0.f);
            }
            // (tmin[e] is FT_SENT when no period reaches epoch e: compare without adding)
            auto live = [&](int e) { return e < Es && tmin[e] < I - i0; };
            auto issue = [&](int e) {
                const int a = (i0 + tmin[e]) & ~1;
                const int len = ((i0 + tmin[e] + tlen[e] + T - a) + 1) & ~1;
                const uint32_t bytes = (uint32_t)len * (uint32_t)sizeof(float2);
                fence_proxy_async();
                mbar_expect_tx(&sm.bar[iss.stage], bytes);
                bulk_load(strips + iss.stage * FT_STRIP, row + a, bytes, &sm.bar[iss.stage]);
                iss.next();
            };
            if (t == 0)
                for (int e = 0; e < FT_NSTAGE - 1 && live(e); ++e) issue(e);
            for (int e = 0; live(e); ++e) {
                if (t == 0 && live(e + FT_NSTAGE - 1)) issue(e + FT_NSTAGE - 1);
                const bool ok = mbar_wait(&sm.bar[con.stage], con.parity);
                const float2 *S = strips + con.stage * FT_STRIP + ((i0 + tmin[e]) & 1) + t;
                con.next();
                const int32_t *de = d + e * GS;
                if (!KAHAN && all_used && full[e] && e == 0) {
                    // every period's epoch-0 offset is 0: one load serves the whole group
                    // (3.5 % faster on the 20-s curve; 1 % slower with compensated sums)
                    float2 v[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = S[r * FT_THREADS];
#pragma unroll
                    for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                        for (int r = 0; r < R; ++r) add2(acc[gg][r], v[r]);
                } else if (all_used && full[e]) {
                    int32_t dv[GS];
                    load_offsets<GS>(de, dv);
#pragma unroll
                    for (int gg = 0; gg < GS; ++gg) {
                        const float2 *src = S + dv[gg];
                        float2 v[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) v[r] = src[r * FT_THREADS];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if constexpr (KAHAN)
                                kahan_add2(acc[gg][r], cmp[gg][r], v[r]);
                            else
                                add2(acc[gg][r], v[r]);
                        }
                    }
                } else {
#pragma unroll
                    for (int gg = 0; gg < GS; ++gg) {
                        const int32_t dg = de[gg];
                        if (dg == FT_SENT || !((use >> gg) & 1u)) continue;
                        const float2 *src = S + dg;
                        float2 v[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) v[r] = src[r * FT_THREADS];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if constexpr (KAHAN)
                                kahan_add2(acc[gg][r], cmp[gg][r], v[r]);
                            else
                                add2(acc[gg][r], v[r]);
                        }
                    }
                }
                if (__syncthreads_or(!ok)) {
                    // a copy did not land in time: record it, drain the ring, stop
                    if (t == 0) {
                        atomicExch(status, CETRA_ETIMEOUT);
                        while (con.n < iss.n) {
                            mbar_wait(&sm.bar[con.stage], con.parity);
                            con.next();
                        }
                    }
                    return false;
                }
            }
            // 2 LR = SA^2 / SB per (period, phase) (a null sum gives NaN, never a maximum);
            // the running max keeps the first (smallest j, then smallest i) of equal values
#pragma unroll
            for (int gg = 0; gg < GS; ++gg) {
                if (!((use >> gg) & 1u)) continue;
                const int nph = sm.nph[g0 + gg];
                const bool whole = i0 + T <= nph;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = i0 + t + r * FT_THREADS;
                    float2 v = acc[gg][r];
                    if constexpr (KAHAN) add2(v, cmp[gg][r]);
                    const float lr2 = v.x * __fdividef(v.x, v.y);
                    if ((whole || i < nph) && lr2 > best_lr[gg]) {
                        best_lr[gg] = lr2;
                        best_at[gg] = (uint32_t)j * (uint32_t)I + (uint32_t)i;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int gg = 0; gg < GS; ++gg)
        if (best_lr[gg] >= 0.0f) {
            const unsigned long long key = make_key(0.5f * best_lr[gg], best_at[gg]);
            if (key > sm.best[g0 + gg][t]) sm.best[g0 + gg][t] = key;
        }
    return true;
}

// A sub-group whose periods all have few phases (nph <= Tp <= T/2, Tp = max(32, nph)):
// the lanes L = t + FT_THREADS r of the block form H = floor(T / Tp) epoch slices of Tp
// phases (lane L: slice L / Tp, phase L % Tp; lanes past H Tp idle); slice h folds epochs
// e = s H + h of super-epoch s, and one bulk copy per super-epoch covers its H epochs. The
// H partial sums of every phase are then added in slice order through shared memory.
// (Strip bound: tmin grows by at most Tp per epoch (o_{e+1} - o_e <= ceil(Ps) <= Tp for the
// period that attains tmin[e]), so a super-epoch needs at most H Tp + spread + 2 <=
// T + spread + 2 cells; the table check keeps spread <= FT_STRIP - FT_T - 8 for this path.)
template <int GS, int R, bool KAHAN>
__device__ bool fold_subgroup_sliced(fold_smem &sm, float2 *strips, const int32_t *tab, int Es,
                                     int g0, int mask_k0, const float2 *__restrict__ ab, int I,
                                     int64_t ld, int J, const double *__restrict__ durations,
                                     const uint8_t *__restrict__ mask, ring &iss, ring &con,
                                     int *__restrict__ status, int Tp) {
    constexpr int T = FT_THREADS * R;
    const int H = T / Tp;
    int slice[R], phase[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int L = threadIdx.x + r * FT_THREADS;
        slice[r] = L / Tp;
        phase[r] = L - slice[r] * Tp;
    }
    const int t = threadIdx.x;
    const int32_t *d = tab;
    const int32_t *tmin = tab + Es * GS;
    const int32_t *tlen = tmin + Es;
    const int32_t *full = tlen + Es;
    float best_lr[GS];
    uint32_t best_at[GS];
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        best_lr[gg] = -1.0f;
        best_at[gg] = 0u;
    }
    auto live_epoch = [&](int e) { return e < Es && tmin[e] < I; };
    for (int j = 0; j < J; ++j) {
        const double D = durations[j];
        unsigned use = 0u;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            const int g = g0 + gg;
            if (sm.E[g] > 0 && D < sm.P[g] && (!mask || mask[(int64_t)(mask_k0 + g) * J + j]))
                use |= 1u << gg;
        }
        if (!use) continue;
        const bool all_used = use == (1u << GS) - 1u;
        const float2 *row = ab + (int64_t)j * ld;
        float2 acc[GS][R];
        float2 cmp[KAHAN ? GS : 1][KAHAN ? R : 1];
#pragma unroll
        for (int gg = 0; gg < GS; ++gg)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[gg][r] = make_float2(0.f, 0.f);
        if constexpr (KAHAN) {
#pragma unroll
            for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                for (int r = 0; r < R; ++r) cmp[gg][r] = make_float2(0.f, 0.f);
        }
        auto issue = [&](int sidx) {
            const int e0 = sidx * H;
            const int a = tmin[e0] & ~1;
            int end = 0;
            for (int h = 0; h < H; ++h)
                if (live_epoch(e0 + h)) end = max(end, tmin[e0 + h] + tlen[e0 + h] + Tp);
            const int len = ((end - a) + 1) & ~1;
            const uint32_t bytes = (uint32_t)len * (uint32_t)sizeof(float2);
            fence_proxy_async();
            mbar_expect_tx(&sm.bar[iss.stage], bytes);
            bulk_load(strips + iss.stage * FT_STRIP, row + a, bytes, &sm.bar[iss.stage]);
            iss.next();
        };
        if (t == 0)
            for (int sidx = 0; sidx < FT_NSTAGE - 1 && live_epoch(sidx * H); ++sidx) issue(sidx);
        for (int sidx = 0; live_epoch(sidx * H); ++sidx) {
            if (t == 0 && live_epoch((sidx + FT_NSTAGE - 1) * H)) issue(sidx + FT_NSTAGE - 1);
            const bool ok = mbar_wait(&sm.bar[con.stage], con.parity);
            const float2 *S = strips + con.stage * FT_STRIP - (tmin[sidx * H] & ~1);
            con.next();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (slice[r] >= H) continue;  // lane past the last whole slice
                const int e = sidx * H + slice[r];
                if (!live_epoch(e)) continue;
                const float2 *src = S + phase[r] + tmin[e];
                const int32_t *de = d + e * GS;
                const bool fast = all_used && full[e];
#pragma unroll
                for (int gg = 0; gg < GS; ++gg) {
                    const int32_t dg = de[gg];
                    if (!fast && (dg == FT_SENT || !((use >> gg) & 1u))) continue;
                    if constexpr (KAHAN)
                        kahan_add2(acc[gg][r], cmp[gg][r], src[dg]);
                    else
                        add2(acc[gg][r], src[dg]);
                }
            }
            if (__syncthreads_or(!ok)) {
                if (t == 0) {
                    atomicExch(status, CETRA_ETIMEOUT);
                    while (con.n < iss.n) {
                        mbar_wait(&sm.bar[con.stage], con.parity);
                        con.next();
                    }
                }
                return false;
            }
        }
        // every copy is consumed: the strip ring is free to hold one period's partial sums
        float2 *part = strips;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            if (!((use >> gg) & 1u)) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 v = acc[gg][r];
                if constexpr (KAHAN) add2(v, cmp[gg][r]);
                part[t + r * FT_THREADS] = v;
            }
            __syncthreads();
            const int nph = sm.nph[g0 + gg];
            for (int phi = t; phi < Tp; phi += FT_THREADS) {
                float2 v = part[phi];
                for (int h = 1; h < H; ++h) add2(v, part[h * Tp + phi]);
                const float lr = 0.5f * (v.x * __fdividef(v.x, v.y));
                if (phi < nph && v.y > 0.0f && lr > best_lr[gg]) {
                    best_lr[gg] = lr;
                    best_at[gg] = (uint32_t)j * (uint32_t)I + (uint32_t)phi;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int gg = 0; gg < GS; ++gg)
        if (best_lr[gg] >= 0.0f) {
            const unsigned long long key = make_key(best_lr[gg], best_at[gg]);
            if (key > sm.best[g0 + gg][t]) sm.best[g0 + gg][t] = key;
        }
    return true;
}

// One period whose offsets do not fit the table: straight from global memory.
__device__ void fold_direct(fold_smem &sm, int g, int k, const float2 *__restrict__ ab, int I,
                            int64_t ld, int J, const double *__restrict__ durations,
                            const uint8_t *__restrict__ mask) {
    const int t = threadIdx.x;
    const double Ps = sm.Ps[g];
    for (int j = 0; j < J; ++j) {
        if (!(durations[j] < sm.P[g])) continue;
        if (mask && !mask[(int64_t)k * J + j]) continue;
        const float2 *row = ab + (int64_t)j * ld;
        for (int i = t; i < sm.nph[g]; i += blockDim.x) {
            float2 acc = make_float2(0.f, 0.f);
            for (int64_t e = 0;; ++e) {
                const int64_t cell = i + epoch_offset(e, Ps);
                if (cell >= I) break;
                add2(acc, row[cell]);
            }
            if (acc.y > 0.0f) {
                const float lr = 0.5f * (acc.x * __fdividef(acc.x, acc.y));
                const unsigned long long key = make_key(lr, (uint32_t)j * (uint32_t)I + (uint32_t)i);
                if (key > sm.best[g][t]) sm.best[g][t] = key;
            }
        }
    }
}

// Per-period metadata of slot t of a group (thread t < FT_G): P, Ps = P/s in t0 steps,
// the number of phases and an upper bound on the epochs with o_e < I.
__device__ __forceinline__ void fold_slot_meta(fold_smem &sm, int t, bool present, double P,
                                               int I, double c, int64_t p, int64_t q) {
    double Ps = 0.0;
    int nph = 0, E = 0;
    if (present) {
        Ps = period_steps(P, c, p, q);
        // a period shorter than one t0 step (or not finite) has no distinct phase: null
        if (Ps >= 1.0 && isfinite(Ps)) {
            const double cph = ceil(Ps);
            nph = cph < (double)I ? (int)cph : I;
            const double eb = floor(__ddiv_rn((double)I + 0.5, Ps)) + 1.0;
            E = eb < 2147483647.0 ? (int)eb : 2147483647;
        }
    } else {
        P = 0.0;
    }
    sm.P[t] = P;
    sm.Ps[t] = Ps;
    sm.nph[t] = nph;
    sm.E[t] = E;
}

// Fold the group whose slot metadata is in `sm` over one (A, B) grid: every sub-group
// (8 -> 4 -> 2 -> 1 periods, as their offsets allow) in turn; the per-thread best key
// of slot g ends in sm.best[g][t]. mask rows are (mask_k0 + g). Returns false if a
// bulk copy timed out (uniform across the block).
template <bool KAHAN, int R>
__device__ bool fold_group(fold_smem &sm, float2 *strips, int32_t *tab,
                           const float2 *__restrict__ ab, int I, int64_t ld, int J,
                           const double *__restrict__ durations, const uint8_t *__restrict__ mask,
                           int mask_k0, ring &iss, ring &con, int *__restrict__ status) {
    const int t = threadIdx.x;
    for (int g = 0; g < FT_G; ++g) sm.best[g][t] = 0ull;
    __syncthreads();
    for (int g0 = 0; g0 < FT_G;) {
        // choose the sub-group [g0, g0 + Gs) and build its table:
        // d [Es][Gs], tmin [Es], tlen [Es], full [Es]
        int Gs = FT_G;
        while (g0 % Gs) Gs >>= 1;
        int Es = 0;
        bool table_ok = false;
        for (;;) {
            Es = 0;
            for (int g = g0; g < g0 + Gs; ++g) Es = max(Es, sm.E[g]);
            if ((int64_t)Es * (Gs + 3) > FT_TABLE) {
                if (Gs > 1) {
                    Gs >>= 1;
                    continue;
                }
                break;  // a single period with too many epochs: no table
            }
            __syncthreads();
            if (t == 0) sm.bad = sm.tight = 0;
            int32_t *tmin = tab + Es * Gs, *tlen = tmin + Es, *full = tlen + Es;
            bool bad = false, tight = false;
            for (int e = t; e < Es; e += blockDim.x) {
                int32_t o[FT_G];
                int32_t mn = FT_SENT, mx = -1, nvalid = 0;
                for (int gg = 0; gg < Gs; ++gg) {
                    const int g = g0 + gg;
                    o[gg] = FT_SENT;
                    if (e < sm.E[g]) {
                        const int64_t v = epoch_offset(e, sm.Ps[g]);
                        if (v < I) o[gg] = (int32_t)v;
                    }
                    if (o[gg] != FT_SENT) {
                        mn = min(mn, o[gg]);
                        mx = max(mx, o[gg]);
                        ++nvalid;
                    }
                }
                for (int gg = 0; gg < Gs; ++gg)
                    tab[e * Gs + gg] = o[gg] == FT_SENT ? FT_SENT : o[gg] - mn;
                tmin[e] = mn;
                tlen[e] = mx - mn;  // < 0 when no period reaches epoch e
                full[e] = nvalid == Gs;
                if (mx - mn > FT_STRIP - FT_T - 2) bad = true;
                if (mx - mn > FT_STRIP - FT_T - 8) tight = true;
            }
            if (bad) sm.bad = 1;
            if (tight) sm.tight = 1;
            __syncthreads();
            if (sm.bad && Gs > 1) {
                Gs >>= 1;
                continue;
            }
            table_ok = !sm.bad;
            break;
        }
        // periods with few phases: fold several epochs at once (epoch slices)
        int nph_sub = 0;
        for (int g = g0; g < g0 + Gs; ++g) nph_sub = max(nph_sub, sm.nph[g]);
        const int tp = max(32, nph_sub);  // phases per epoch slice
        const bool sliced = table_ok && !sm.tight && nph_sub > 0 &&
                            2 * tp <= FT_THREADS * R;
        bool ok = true;
        if (!table_ok) {
            fold_direct(sm, g0, mask_k0 + g0, ab, I, ld, J, durations, mask);
        } else if (sliced) {
            if (Gs == 8)
                ok = fold_subgroup_sliced<8, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I,
                                                       ld, J, durations, mask, iss, con, status,
                                                       tp);
            else if (Gs == 4)
                ok = fold_subgroup_sliced<4, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I,
                                                       ld, J, durations, mask, iss, con, status,
                                                       tp);
            else if (Gs == 2)
                ok = fold_subgroup_sliced<2, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I,
                                                       ld, J, durations, mask, iss, con, status,
                                                       tp);
            else
                ok = fold_subgroup_sliced<1, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I,
                                                       ld, J, durations, mask, iss, con, status,
                                                       tp);
        } else if (Gs == 8) {
            ok = fold_subgroup<8, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I, ld, J,
                                            durations, mask, iss, con, status);
        } else if (Gs == 4) {
            ok = fold_subgroup<4, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I, ld, J,
                                            durations, mask, iss, con, status);
        } else if (Gs == 2) {
            ok = fold_subgroup<2, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I, ld, J,
                                            durations, mask, iss, con, status);
        } else {
            ok = fold_subgroup<1, R, KAHAN>(sm, strips, tab, Es, g0, mask_k0, ab, I, ld, J,
                                            durations, mask, iss, con, status);
        }
        if (!ok) return false;
        g0 += Gs;
    }
    return true;
}

__device__ __forceinline__ void fold_init_barriers(fold_smem &sm) {
    if (threadIdx.x == 0) {
        for (int st = 0; st < FT_NSTAGE; ++st) mbar_init(&sm.bar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

template <bool KAHAN>
__global__ void __launch_bounds__(FT_THREADS, FT_MIN_BLOCKS)
fold_tma_kernel(const float2 *__restrict__ ab, int I, int64_t ld, int J,
                const double *__restrict__ durations, const double *__restrict__ periods, int K,
                const uint8_t *__restrict__ mask, double c, int64_t p, int64_t q,
                unsigned long long *__restrict__ keys, int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *strips = reinterpret_cast<float2 *>(smem_raw);                      // [NSTAGE][STRIP]
    int32_t *tab = reinterpret_cast<int32_t *>(strips + FT_NSTAGE * FT_STRIP);  // FT_TABLE
    __shared__ fold_smem sm;
    const int t = threadIdx.x;
    fold_init_barriers(sm);
    ring iss, con;
    const int ngroups = (K + FT_G - 1) / FT_G;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int k0 = grp * FT_G;
        __syncthreads();  // the previous group is done with the shared tables
        if (t < FT_G) fold_slot_meta(sm, t, k0 + t < K, k0 + t < K ? periods[k0 + t] : 0.0, I, c, p, q);
        if (!fold_group<KAHAN, KAHAN ? FT_R / 2 : FT_R>(sm, strips, tab, ab, I, ld, J, durations,
                                                         mask, k0, iss, con, status))
            return;  // uniform: every thread saw the same vote
        for (int g = 0; g < FT_G; ++g) {
            const unsigned long long v = block_max_key(sm.best[g][t], sm.red);
            if (t == 0 && k0 + g < K) keys[k0 + g] = v;
        }
    }
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
__global__ void logl0_kernel(const float *__restrict__ wy, const float *__restrict__ w, int64_t n,
                             double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double W = (double)w[k];
        if (!(W > 0.0)) continue;
        const double y = (double)wy[k] / W;
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
__device__ __forceinline__ int csr_find(const int64_t *__restrict__ off, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Period k of a batch curve: pmin * ratio^k, ratio^k by LSB-first square-and-multiply.
__device__ __forceinline__ double batch_period(double pmin, double ratio, int64_t k) {
    double x = 1.0, b = ratio;
    while (k) {
        if (k & 1) x = __dmul_rn(x, b);
        b = __dmul_rn(b, b);
        k >>= 1;
    }
    return __dmul_rn(pmin, x);
}

// Sec. 2.1.1 for every point of every curve (curve found from the point index).
__global__ void batch_resample_kernel(const double *__restrict__ time,
                                      const float *__restrict__ flux,
                                      const float *__restrict__ err, int64_t n,
                                      const int64_t *__restrict__ pt_off, int n_curves,
                                      const batch_curve *__restrict__ curves, double c,
                                      int64_t n_pad, int flux_is_offset, float *__restrict__ wy,
                                      float *__restrict__ w) {
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
        atomicAdd(&wy[bin], wk * yk);
        atomicAdd(&w[bin], wk);
    }
}

// Sec. 2.2 for every curve: x-blocks enumerate the t0 tiles of all curves.
template <int RB, bool KAHAN>
__global__ void __launch_bounds__(128, 4)
batch_linear_kernel(const int64_t *__restrict__ tile_off, int n_curves,
                    const batch_curve *__restrict__ curves, const float *__restrict__ wy,
                    const float *__restrict__ w, const float2 *__restrict__ tables,
                    const int32_t *__restrict__ win_a, const int32_t *__restrict__ win_padlen,
                    const int64_t *__restrict__ win_off, int p, int q, int kc_max,
                    const int32_t *__restrict__ order, float2 *__restrict__ ab) {
    const int cidx = csr_find(tile_off, n_curves, blockIdx.x);
    const batch_curve cv = curves[cidx];
    if (cv.I <= 0) return;
    if (p == 1)
        linear_block<RB, KAHAN, 1>((int)(blockIdx.x - tile_off[cidx]), order[blockIdx.y],
                                   wy + cv.grid_off, w + cv.grid_off, cv.n_grid, tables, win_a,
                                   win_padlen, win_off, p, q, cv.I, cv.ld, kc_max,
                                   ab + cv.ab_off, nullptr, nullptr, nullptr);
    else
        linear_block<RB, KAHAN, 0>((int)(blockIdx.x - tile_off[cidx]), order[blockIdx.y],
                                   wy + cv.grid_off, w + cv.grid_off, cv.n_grid, tables, win_a,
                                   win_padlen, win_off, p, q, cv.I, cv.ld, kc_max,
                                   ab + cv.ab_off, nullptr, nullptr, nullptr);
}

// Sec. 2.3 for every curve: persistent blocks drain a queue of (curve, group of FT_G
// periods) items; each group's best per period goes into the curve's key
// (LR bits, inverted period index: the largest LR wins, ties to the smallest period index).
template <bool KAHAN, int R>
__global__ void __launch_bounds__(FT_THREADS, FT_MIN_BLOCKS)
batch_fold_kernel(const float2 *__restrict__ ab, const batch_curve *__restrict__ curves,
                  const int64_t *__restrict__ group_off, int n_curves, int64_t n_items, int J,
                  const double *__restrict__ durations, double c, int64_t p, int64_t q,
                  int *__restrict__ queue, unsigned long long *__restrict__ period_keys,
                  unsigned long long *__restrict__ curve_keys, int *__restrict__ status,
                  const int64_t *__restrict__ item_list,
                  const unsigned long long *__restrict__ n_items_dev) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the queue length: n_items, or the count a device-side selection left (capped by n_items)
    if (n_items_dev) n_items = min(n_items, (int64_t)*n_items_dev);
    float2 *strips = reinterpret_cast<float2 *>(smem_raw);
    int32_t *tab = reinterpret_cast<int32_t *>(strips + FT_NSTAGE * FT_STRIP);
    __shared__ fold_smem sm;
    __shared__ int s_item;
    const int t = threadIdx.x;
    fold_init_barriers(sm);
    ring iss, con;
    for (;;) {
        __syncthreads();  // the previous item is done with the shared state
        if (t == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        if (s_item >= n_items) break;
        // queue position -> work item: the position itself, or the caller's list entry
        const int64_t item = item_list ? item_list[s_item] : (int64_t)s_item;
        const int cidx = csr_find(group_off, n_curves, item);
        const batch_curve cv = curves[cidx];
        const int k0 = (int)(item - group_off[cidx]) * FT_G;
        if (t < FT_G) {
            const bool present = k0 + t < cv.n_periods;
            fold_slot_meta(sm, t, present, present ? batch_period(cv.pmin, cv.ratio, k0 + t) : 0.0,
                           cv.I, c, p, q);
        }
        if (!fold_group<KAHAN, R>(sm, strips, tab, ab + cv.ab_off, cv.I, cv.ld, J, durations,
                                  nullptr, 0, iss, con, status))
            return;  // uniform
        for (int g = 0; g < FT_G; ++g) {
            const unsigned long long v = block_max_key(sm.best[g][t], sm.red);
            if (t == 0 && k0 + g < cv.n_periods) {
                period_keys[cv.per_off + k0 + g] = v;
                if (v != 0ull)
                    atomicMax(&curve_keys[cidx],
                              (v & 0xFFFFFFFF00000000ull) |
                                  (unsigned long long)(0xFFFFFFFFu - (uint32_t)(k0 + g)));
            }
        }
    }
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

size_t fold_smem_bytes() {
    return (size_t)FT_NSTAGE * FT_STRIP * sizeof(float2) + (size_t)FT_TABLE * sizeof(int32_t);
}

// ============================================================================================
// launchers

cudaError_t launch_resample(cetra_ctx *ctx, const cetra_plan *plan, const double *time,
                            const float *flux, const float *err, int64_t n, float *wy, float *w) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    blocks = blocks > (int64_t)ctx->num_sms * 16 ? (int64_t)ctx->num_sms * 16 : blocks;
    prof_mark(ctx, KID_RESAMPLE, true);
    resample_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(
        time, flux, err, n, plan->t_ref, plan->cadence, plan->n_pad, plan->n_grid,
        plan->flux_is_offset, wy, w);
    prof_mark(ctx, KID_RESAMPLE, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t linear_configure(cetra_plan *plan, const cetra_ctx *ctx) {
    const int p = (int)plan->p;
    const size_t budget = 100 * 1024;  // keeps two blocks resident per SM at the largest shape
    const int unit = p * LIN_RB;
    int kc = (2304 / unit) * unit;
    if (kc < unit) kc = unit;
    if (plan->max_padlen > 0 && kc > plan->max_padlen) kc = plan->max_padlen;
    int threads = 128;
    auto bytes = [&](int th, int k) { return ((size_t)p * th * LIN_RB + 2 * (size_t)k) * sizeof(float2); };
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
    // the fold's strip ring and offset table (dynamic) exceed the default 48 KiB
    for (auto fn : {fold_tma_kernel<false>, fold_tma_kernel<true>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fold_smem_bytes());
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_linear(cetra_ctx *ctx, const cetra_plan *plan, const float *wy, const float *w,
                          float2 *ab, float *depth, float *var, float *dlogl) {
    const int64_t I = plan->n_t0, q = plan->q;
    const int64_t Umax = (I + q - 1) / q;
    const int64_t UT = (int64_t)plan->lin_threads * LIN_RB;
    const int64_t gx = (Umax + UT - 1) / UT;
    if (gx == 0) return cudaSuccess;
    dim3 grid((unsigned)gx, (unsigned)(plan->J * q));
    prof_mark(ctx, KID_LINEAR, true);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? linear_kernel<LIN_RB, true>
                                                    : linear_kernel<LIN_RB, false>;
    kern<<<grid, plan->lin_threads, plan->lin_smem, ctx->stream>>>(
        wy, w, plan->n_grid, plan->d_tables, plan->d_win_a, plan->d_win_padlen, plan->d_win_off,
        (int)plan->p, (int)q, I, plan->ab_ld, plan->lin_kc, plan->d_lin_order, ab, depth, var,
        dlogl);
    prof_mark(ctx, KID_LINEAR, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_fold(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                        const double *periods, int K, const uint8_t *mask,
                        unsigned long long *keys, int *status) {
    if (K <= 0) return cudaSuccess;
    const int ngroups = (K + FT_G - 1) / FT_G;
    prof_mark(ctx, KID_FOLD, true);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? fold_tma_kernel<true> : fold_tma_kernel<false>;
    kern<<<ngroups, FT_THREADS, fold_smem_bytes(), ctx->stream>>>(
        ab, (int)plan->n_t0, plan->ab_ld, plan->J, plan->d_durations, periods, K, mask,
        plan->cadence, plan->p, plan->q, keys, status);
    prof_mark(ctx, KID_FOLD, false);
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

cudaError_t launch_logl0(cetra_ctx *ctx, const cetra_plan *plan, const float *wy, const float *w,
                         double *out) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), ctx->stream);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    int64_t blocks = (plan->n_grid + threads - 1) / threads;
    if (blocks > (int64_t)ctx->num_sms * 4) blocks = (int64_t)ctx->num_sms * 4;
    if (blocks < 1) blocks = 1;
    prof_mark(ctx, KID_LOGL0, true);
    logl0_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(wy, w, plan->n_grid, out);
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
                                  const batch_curve *curves, float *wy, float *w) {
    if (n_points <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n_points + threads - 1) / threads;
    if (blocks > (int64_t)num_sms * 32) blocks = (int64_t)num_sms * 32;
    batch_resample_kernel<<<(unsigned)blocks, threads, 0, stream>>>(
        time, flux, err, n_points, pt_offsets, n_curves, curves, plan->cadence, plan->n_pad,
        plan->flux_is_offset, wy, w);
    return cudaGetLastError();
}

cudaError_t launch_batch_linear(cudaStream_t stream, const cetra_plan *plan, int threads,
                                const int64_t *tile_off, int n_curves, int64_t n_tiles,
                                const batch_curve *curves, const float *wy, const float *w,
                                float2 *ab) {
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 2147483647) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)n_tiles, (unsigned)(plan->J * plan->q));
    const size_t smem = ((size_t)plan->p * threads * LIN_RB + 2 * (size_t)plan->lin_kc) *
                        sizeof(float2);
    auto kern = plan->precision == CETRA_FP32_KAHAN ? batch_linear_kernel<LIN_RB, true>
                                                    : batch_linear_kernel<LIN_RB, false>;
    kern<<<grid, threads, smem, stream>>>(tile_off, n_curves, curves, wy, w, plan->d_tables,
                                          plan->d_win_a, plan->d_win_padlen, plan->d_win_off,
                                          (int)plan->p, (int)plan->q, plan->lin_kc,
                                          plan->d_lin_order, ab);
    return cudaGetLastError();
}

// Fold variants the autotuner chooses from: phases per thread (FT_R or FT_R / 2).
int batch_fold_variants() { return 2; }
int batch_fold_blocks_per_sm(int) { return FT_MIN_BLOCKS; }

cudaError_t launch_batch_fold(cudaStream_t stream, int blocks, int variant, const cetra_plan *plan,
                              const float2 *ab, const batch_curve *curves,
                              const int64_t *group_off, int n_curves, int64_t n_items,
                              int *queue, unsigned long long *period_keys,
                              unsigned long long *curve_keys, int *status,
                              const int64_t *item_list, const unsigned long long *n_items_dev) {
    if (n_items <= 0) return cudaSuccess;
    auto kern = batch_fold_kernel<false, FT_R>;
    if (plan->precision == CETRA_FP32_KAHAN)
        kern = batch_fold_kernel<true, FT_R / 2>;
    else if (variant == 1)
        kern = batch_fold_kernel<false, FT_R / 2>;
    kern<<<blocks, FT_THREADS, fold_smem_bytes(), stream>>>(
        ab, curves, group_off, n_curves, n_items, plan->J, plan->d_durations, plan->cadence,
        plan->p, plan->q, queue, period_keys, curve_keys, status, item_list, n_items_dev);
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
    const size_t lin_max = ((size_t)plan->p * 128 * LIN_RB + 2 * (size_t)plan->lin_kc) * sizeof(float2);
    for (auto fn : {batch_linear_kernel<LIN_RB, false>, batch_linear_kernel<LIN_RB, true>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)lin_max);
        if (e != cudaSuccess) return e;
    }
    for (auto fn : {batch_fold_kernel<false, FT_R>, batch_fold_kernel<false, FT_R / 2>,
                    batch_fold_kernel<true, FT_R / 2>}) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fold_smem_bytes());
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
