// sm_103a kernels of the CETRA hot path.
//
//   resample_kernel   Sec. 2.1.1  nearest-grid-point scatter of (W y, W), W = 1/sigma^2
//   linear_kernel     Sec. 2.2    per (duration, t0): A = sum m W y, B = sum m^2 W over the
//                                 window; depth = A/B, var = 1/B, dlogl = A^2/(2B)
//   fold_group_kernel Sec. 2.3    per group of periods: sum A and B over the epoch cells of
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
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(acc)), "l"(pack2(v)));
    acc = unpack2(d);
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
template <int RB>
__global__ void __launch_bounds__(128)
linear_kernel(const float *__restrict__ wy, const float *__restrict__ w, int64_t n_grid,
              const float2 *__restrict__ tables, const int32_t *__restrict__ win_a,
              const int32_t *__restrict__ win_padlen, const int64_t *__restrict__ win_off, int p,
              int q, int64_t I, int kc_max, float2 *__restrict__ ab, float *__restrict__ depth,
              float *__restrict__ var, float *__restrict__ dlogl) {
    extern __shared__ float2 smem[];
    const int nthr = blockDim.x;
    const int t = threadIdx.x;
    const int jr = blockIdx.y;
    const int j = jr / q, r = jr % q;
    const int64_t U = (r < I) ? (I - r + q - 1) / q : 0;
    const int64_t UT = (int64_t)nthr * RB;
    const int64_t u0 = (int64_t)blockIdx.x * UT;
    if (u0 >= U) return;
    const int padlen = win_padlen[jr];
    const int64_t a0 = (int64_t)win_a[jr] + (int64_t)p * u0;
    const float2 *tab = tables + win_off[jr];
    float2 *st = smem;           // [kc_max] template chunk (m, m^2)
    float2 *sd = smem + kc_max;  // [p*UT + kc_max] grid span (W y, W)

    // Blocked summation: `acc` collects at most LIN_SUB * RB terms before it is
    // folded into `tot`, so the FP32 rounding error grows with the block length
    // plus the number of blocks instead of with the window length.
    float2 acc[RB], tot[RB];
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) acc[rr] = tot[rr] = make_float2(0.f, 0.f);

    for (int kc0 = 0; kc0 < padlen; kc0 += kc_max) {
        const int kcl = min(kc_max, padlen - kc0);
        __syncthreads();
        for (int idx = t; idx < kcl; idx += nthr) st[idx] = tab[kc0 + idx];
        const int64_t base = a0 + kc0;
        const int dl = (int)(p * UT) + kcl;
        for (int idx = t; idx < dl; idx += nthr) {
            const int64_t n = base + idx;
            float2 v = make_float2(0.f, 0.f);
            if (n >= 0 && n < n_grid) v = make_float2(wy[n], w[n]);
            sd[idx] = v;
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
                        for (int rr = 0; rr < RB; ++rr) fma2(acc[rr], mm, buf[(s + rr) % RB]);
                        buf[s] = V[p * (k1 + RB)];
                    }
                }
#pragma unroll
                for (int rr = 0; rr < RB; ++rr) {
                    add2(tot[rr], acc[rr]);
                    acc[rr] = make_float2(0.f, 0.f);
                }
            }
        }
    }
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) acc[rr] = tot[rr];

#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
        const int64_t u = u0 + (int64_t)t * RB + rr;
        if (u >= U) break;
        const int64_t i = r + (int64_t)q * u;
        const int64_t idx = (int64_t)j * I + i;
        const float A = acc[rr].x, B = acc[rr].y;
        ab[idx] = acc[rr];
        const bool ok = B > 0.0f;
        if (depth) depth[idx] = ok ? A / B : __int_as_float(0x7fc00000);
        if (var) var[idx] = ok ? 1.0f / B : __int_as_float(0x7fc00000);
        if (dlogl) dlogl[idx] = ok ? 0.5f * (A * (A / B)) : __int_as_float(0x7fc00000);
    }
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
// Sec. 2.3 periodic search, FOLD_G periods per block. Neighbouring trial periods
// gather nearly the same epoch cells (their offsets differ by a few cells), so a
// thread folds its phase i for all FOLD_G periods together: the first period's
// loads bring the cache lines into L1 and the others hit them. The epoch offsets
// of the group live in shared memory as [e][g]. A group whose offsets do not fit
// is folded one period at a time (table of that period only), and a period
// whose own table does not fit computes its offsets on the fly in FP64.
#ifndef FOLD_MIN_BLOCKS
#define FOLD_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(FOLD_THREADS, FOLD_MIN_BLOCKS)
fold_group_kernel(const float2 *__restrict__ ab, int64_t I, int J,
                  const double *__restrict__ durations, const double *__restrict__ periods, int K,
                  const uint8_t *__restrict__ mask, double c, int64_t p, int64_t q,
                  unsigned long long *__restrict__ keys) {
    extern __shared__ int32_t off[];  // FOLD_TABLE entries
    __shared__ unsigned long long red[FOLD_THREADS / 32];
    __shared__ unsigned long long s_best[FOLD_G][FOLD_THREADS];  // per-thread best key per period
    __shared__ double s_P[FOLD_G], s_Ps[FOLD_G];
    __shared__ int64_t s_nph[FOLD_G];
    __shared__ int s_E[FOLD_G];
    const int t = threadIdx.x;
    const int ngroups = (K + FOLD_G - 1) / FOLD_G;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int k0 = grp * FOLD_G;
        __syncthreads();  // the previous group is done with the shared tables
        if (t < FOLD_G) {
            const int k = k0 + t;
            double P = 0.0, Ps = 0.0;
            int64_t nph = 0;
            int E = 0;
            if (k < K) {
                P = periods[k];
                Ps = period_steps(P, c, p, q);
                // a period shorter than one t0 step (or not finite) has no distinct phase: null
                if (Ps >= 1.0 && isfinite(Ps)) {
                    const double cph = ceil(Ps);
                    nph = cph < (double)I ? (int64_t)cph : I;
                    const double eb = floor(__ddiv_rn((double)I + 0.5, Ps)) + 1.0;
                    E = eb < 2147483647.0 ? (int)eb : 2147483647;
                }
            }
            s_P[t] = P;
            s_Ps[t] = Ps;
            s_nph[t] = nph;
            s_E[t] = E;
        }
        __syncthreads();
        int Emax = 0;
        int64_t nphmax = 0;
#pragma unroll
        for (int g = 0; g < FOLD_G; ++g) {
            Emax = max(Emax, s_E[g]);
            nphmax = max(nphmax, s_nph[g]);
        }
        const bool grouped = (int64_t)Emax * FOLD_G <= FOLD_TABLE;
        if (grouped) {
            for (int idx = t; idx < Emax * FOLD_G; idx += blockDim.x) {
                const int e = idx / FOLD_G, g = idx % FOLD_G;
                int32_t o = INT32_MAX;
                if (e < s_E[g]) {
                    const int64_t v = epoch_offset(e, s_Ps[g]);
                    if (v < I) o = (int32_t)v;
                }
                off[idx] = o;
            }
        }
        __syncthreads();

#pragma unroll
        for (int g = 0; g < FOLD_G; ++g) s_best[g][t] = 0ull;

        if (grouped) {
            for (int j = 0; j < J; ++j) {
                const double D = durations[j];
                unsigned use = 0u;
#pragma unroll
                for (int g = 0; g < FOLD_G; ++g) {
                    const int k = k0 + g;
                    if (s_E[g] > 0 && D < s_P[g] && (!mask || mask[(int64_t)k * J + j]))
                        use |= 1u << g;
                }
                if (!use) continue;
                const float2 *row = ab + (int64_t)j * I;
                for (int64_t i = t; i < nphmax; i += blockDim.x) {
                    unsigned act = 0u;
#pragma unroll
                    for (int g = 0; g < FOLD_G; ++g)
                        if (((use >> g) & 1u) && i < s_nph[g]) act |= 1u << g;
                    float2 acc[FOLD_G];
#pragma unroll
                    for (int g = 0; g < FOLD_G; ++g) acc[g] = make_float2(0.f, 0.f);
                    for (int e = 0; e < Emax && act; ++e) {
                        const int4 oa = *reinterpret_cast<const int4 *>(&off[e * FOLD_G]);
                        const int4 ob = *reinterpret_cast<const int4 *>(&off[e * FOLD_G + 4]);
                        const int o[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
                        unsigned live = 0u;
#pragma unroll
                        for (int g = 0; g < FOLD_G; ++g) {
                            if (((act >> g) & 1u) && i + (int64_t)o[g] < I) {
                                add2(acc[g], row[i + o[g]]);
                                live |= 1u << g;
                            }
                        }
                        act = live;  // offsets grow with e: a period past the end stays past it
                    }
#pragma unroll
                    for (int g = 0; g < FOLD_G; ++g) {
                        if (acc[g].y > 0.0f && ((use >> g) & 1u) && i < s_nph[g]) {
                            const float lr = 0.5f * (acc[g].x * (acc[g].x / acc[g].y));
                            const unsigned long long key =
                                make_key(lr, (uint32_t)((int64_t)j * I + i));
                            if (key > s_best[g][t]) s_best[g][t] = key;
                        }
                    }
                }
            }
        } else {
            // one period at a time: its own offsets in the table when they fit
#pragma unroll
            for (int g = 0; g < FOLD_G; ++g) {
                const int E = s_E[g];
                const double Ps = s_Ps[g];
                const bool tab = E <= FOLD_TABLE;
                __syncthreads();
                if (tab)
                    for (int e = t; e < E; e += blockDim.x) {
                        const int64_t v = epoch_offset(e, Ps);
                        off[e] = v < I ? (int32_t)v : INT32_MAX;
                    }
                __syncthreads();
                if (E == 0) continue;
                const int k = k0 + g;
                for (int j = 0; j < J; ++j) {
                    if (!(durations[j] < s_P[g])) continue;
                    if (mask && !mask[(int64_t)k * J + j]) continue;
                    const float2 *row = ab + (int64_t)j * I;
                    for (int64_t i = t; i < s_nph[g]; i += blockDim.x) {
                        float2 acc = make_float2(0.f, 0.f);
                        if (tab) {
                            for (int e = 0; e < E; ++e) {
                                const int o = off[e];
                                if (i + (int64_t)o >= I) break;
                                add2(acc, row[i + o]);
                            }
                        } else {
                            for (int64_t e = 0;; ++e) {
                                const int64_t cell = i + epoch_offset(e, Ps);
                                if (cell >= I) break;
                                add2(acc, row[cell]);
                            }
                        }
                        if (acc.y > 0.0f) {
                            const float lr = 0.5f * (acc.x * (acc.x / acc.y));
                            const unsigned long long key =
                                make_key(lr, (uint32_t)((int64_t)j * I + i));
                            if (key > s_best[g][t]) s_best[g][t] = key;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int g = 0; g < FOLD_G; ++g) {
            const unsigned long long v = block_max_key(s_best[g][t], red);
            if (t == 0 && k0 + g < K) keys[k0 + g] = v;
        }
    }
}

// --------------------------------------------------------------------------------------------
// Sec. 2.3: the per-period winner, re-summed in FP64 from the FP32 grid.
__global__ void finalize_kernel(const float2 *__restrict__ ab, int64_t I,
                                const double *__restrict__ durations,
                                const double *__restrict__ periods, int K,
                                const unsigned long long *__restrict__ keys, double t_ref, double c,
                                int64_t p, int64_t q, int64_t n_pad, double *dlogl, double *t0,
                                double *dur, double *depth, double *var, int64_t *oi, int32_t *oj) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const unsigned long long key = keys[k];
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (key == 0ull) {
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
    const float2 *row = ab + j * I;
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

}  // namespace

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
    cudaError_t e = cudaFuncSetAttribute(linear_kernel<LIN_RB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan->lin_smem);
    if (e != cudaSuccess) return e;
    // the grouped fold's offset table (dynamic) plus its per-thread keys (static) exceed 48 KiB
    return cudaFuncSetAttribute(fold_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(FOLD_TABLE * sizeof(int32_t)));
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
    linear_kernel<LIN_RB><<<grid, plan->lin_threads, plan->lin_smem, ctx->stream>>>(
        wy, w, plan->n_grid, plan->d_tables, plan->d_win_a, plan->d_win_padlen, plan->d_win_off,
        (int)plan->p, (int)q, I, plan->lin_kc, ab, depth, var, dlogl);
    prof_mark(ctx, KID_LINEAR, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_fold(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                        const double *periods, int K, const uint8_t *mask,
                        unsigned long long *keys) {
    if (K <= 0) return cudaSuccess;
    prof_mark(ctx, KID_FOLD, true);
    const int ngroups = (K + FOLD_G - 1) / FOLD_G;
    fold_group_kernel<<<ngroups, FOLD_THREADS, FOLD_TABLE * sizeof(int32_t), ctx->stream>>>(
        ab, plan->n_t0, plan->J, plan->d_durations, periods, K, mask, plan->cadence, plan->p,
        plan->q, keys);
    prof_mark(ctx, KID_FOLD, false);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_finalize(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                            const double *periods, int K, const unsigned long long *keys,
                            double *dlogl, double *t0, double *dur, double *depth, double *var,
                            int64_t *oi, int32_t *oj) {
    if (K <= 0) return cudaSuccess;
    const int threads = 128;
    prof_mark(ctx, KID_FINALIZE, true);
    finalize_kernel<<<(K + threads - 1) / threads, threads, 0, ctx->stream>>>(
        ab, plan->n_t0, plan->d_durations, periods, K, keys, plan->t_ref, plan->cadence, plan->p,
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
