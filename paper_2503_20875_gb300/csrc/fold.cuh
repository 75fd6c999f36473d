// Sec. 2.3 periodic search on sm_103a: the fold of the linear grid over trial periods with a
// common depth (Eq. 3, Eq. 4) and the in-kernel maximum per period.
//
// With A = sum m W y and B = sum m^2 W per window (Sec. 2.2), Eq. 4 at the common depth
// Z = sum_e A_e / sum_e B_e is (sum_e A_e)^2 / (2 sum_e B_e), so the fold only sums (A, B)
// pairs over the epoch cells i + o_e, o_e = floor(e P / s + 1/2) (the nearest t0 point of
// epoch e, FP64). A null window is (0, 0) and drops out of the sums.
//
// Device code shared by the single-curve fold (fold.cu) and the batched fold (fold_batch.cu).
//
// Work: one block per group of FT_G neighbouring trial periods and a chunk of durations (one
// duration for grids larger than the L2). Neighbouring periods read nearly the same cells, so for a tile of
// T phases and an epoch e the block copies the union of the cells its periods need,
// [i0 + min_g o_e(g), i0 + max_g o_e(g) + T), into shared memory with one bulk copy and every
// period reads its cells from there.
//
// Block: FT_THREADS consumer threads and one producer warp. The producer issues the bulk
// copies into a ring of strips in shared memory; each strip has a "full" barrier (completed
// by the copy's byte count) and an "empty" barrier (completed when every consumer thread has
// read it). Consumers wait only for the strip they read next, so there is no block-wide
// barrier per epoch; warps drift freely and the shared-memory pipe stays busy. The ring's
// strips are as long as the sub-group being folded needs (a tile plus the widest spread of its
// offsets), so narrow groups get up to FT_NSTAGE strips in flight. Consumer thread c owns
// phases i0 + c + r FT_THREADS (r < R) of every period of the sub-group and keeps their
// (A, B) sums in registers as packed FP32 pairs: one 8-byte shared load and one packed add
// per cell read.
//
// Epoch table: per sub-group the epoch offsets are computed once in FP64 into shared memory
// as byte offsets of each period's first cell within the epoch's strip (32-bit when the
// table fits, else 16-bit), plus the smallest and largest offset of the epoch (the strip's
// extent). Groups whose table does not fit, or whose offsets spread wider than a strip
// allows, are split 8 -> 4 -> 2 -> 1; a single period whose table does not fit is folded
// straight from global memory. The last tile of each duration row folds only the rows of
// FT_THREADS phases that hold a phase. Periods with few phases (at most T/2) fold several
// durations per tile when the work item has several (duration-packed path), else several
// epochs per strip (epoch slices).
//
// Bounded waits: every barrier wait gives up after FT_WAIT_CYCLES; the thread records
// CETRA_ETIMEOUT in the status word and raises the block's abort flag, after which no thread
// waits or issues a copy any more: every thread runs on to the same block barriers (none
// leaves the kernel early, so every block barrier completes), the producer waits (bounded)
// for the copies it still has in flight, and the block exits. The finalize kernel then writes
// NaN for every period.
#pragma once

#include <cfloat>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace {

// ---------------------------------------------------------------------------------------------
// Packed (A, B) pairs and shared-memory access by 32-bit address.

// One (A, B) cell as a packed FP32 pair (A in the low half); sums stay packed, so no register
// moves are needed around the packed adds.
__device__ __forceinline__ uint64_t lds_pair(uint32_t addr) {
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// v[k] = the pair at addr + k FT_THREADS * 8 (k < R): the rows of R phases a thread owns in a
// strip, with the row step as an immediate offset of each load.
template <int K, int R>
__device__ __forceinline__ void lds_rows(uint64_t (&v)[R], uint32_t addr) {
    if constexpr (K < R) {
        asm volatile("ld.shared.b64 %0, [%1+%2];"
                     : "=l"(v[K])
                     : "r"(addr), "n"(K * FT_THREADS * (int)sizeof(float2)));
        lds_rows<K + 1, R>(v, addr);
    }
}

__device__ __forceinline__ int32_t lds_s32(uint32_t addr) {
    int32_t v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// acc += v on packed FP32 pairs.
__device__ __forceinline__ void add_pair(uint64_t &acc, uint64_t v) {
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc) : "l"(v));
}

// a + b on packed FP32 pairs.
__device__ __forceinline__ uint64_t sum_pair(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Kahan-compensated s += v on packed pairs; nc holds minus the running compensation:
// y = v + nc, t = s + y, nc = y - (t - s), s = t.
__device__ __forceinline__ void kahan_add_pair(uint64_t &s, uint64_t &nc, uint64_t v) {
    uint64_t y, t, d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(y) : "l"(v), "l"(nc));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(s), "l"(y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(t), "l"(s));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(nc) : "l"(y), "l"(d));
    s = t;
}

__device__ __forceinline__ void split_pair(uint64_t v, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}

// Block-wide barrier that threads may reach from different call sites (the producer warp and
// the consumer warps run different loops; the non-aligned form allows that).
__device__ __forceinline__ void block_sync() { asm volatile("barrier.sync 0;" ::: "memory"); }

// One arrival on a barrier (release of this thread's earlier shared-memory reads).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Candidate test of the epilogue: the exact comparison of a window's 2 LR = x^2 / y with the
// running best b is x * __fdividef(x, y) > b, whose left side has a relative error below
// 2^-21. With h = b (1 - 2^-14) and q = h y (each rounded once), fma(x, x, -q) > 0 (the exact
// x^2 - q, rounded) holds whenever the exact comparison does (for b <= 0 trivially, for b > 0
// by the margin), so a tile whose largest fma(x, x, -q) is not positive has no new maximum;
// otherwise the exact comparison runs over the tile's windows in order, and decides as before.
constexpr float kCandidate = 1.0f - 1.0f / 16384.0f;

// ---------------------------------------------------------------------------------------------
// Shared state.

// The work item a block folds: one (A, B) grid, durations [jlo, jhi), the group's mask rows.
// Kept in shared memory so that it takes no registers in the hot loops.
struct fold_item {
    const float2 *ab;
    const double *durations;
    const uint8_t *mask;  // [K][J] or NULL; rows mask_k0 + g
    int *status;
    int64_t ld;
    int I, J, jlo, jhi, mask_k0;
    int gmax;  // largest sub-group (periods folded together), a power of two <= FT_G
};

struct fold_smem {
    uint64_t full[FT_NSTAGE];        // strip landed: the producer's arrival + the copy's bytes
    uint64_t empty[FT_NSTAGE];       // strip read: one arrival per consumer thread
    unsigned long long best[FT_G];   // best key of each slot of the group
    double P[FT_G], Ps[FT_G];        // period (days) and period in t0 steps
    int nph[FT_G], E[FT_G];          // phases, and an upper bound on the epochs with o_e < I
    int bad, tight;                  // table votes: spread too wide for the main / sliced path
    int spread;                      // widest spread of the table's epochs (cells)
    int abort;                       // a bounded wait gave up: no more waits or copies
    int pack_n;                      // duration-packed path: durations in the list below
    int16_t pack_j[FT_PACK_MAXJ];    // the durations at which some period of the sub-group
    uint8_t pack_use[FT_PACK_MAXJ];  // is folded (ascending), and period_use of each
    fold_item it;
};

// The strip ring as both sides see it. A sub-group uses ns strips of `bytes` each; strip s
// has been filled f_s times so far, and bit s of `par` is f_s mod 2: its next fill completes
// phase parity (par >> s) & 1 of full[s] and needs phase f_s - 1 of empty[s] to be complete.
// The producer and every consumer step through the same sequence of strips.
struct ring {
    uint32_t stage = 0, ns = 1, bytes = 0, par = 0;
    __device__ __forceinline__ void start(uint32_t nstages, uint32_t stage_bytes) {
        stage = 0;
        ns = nstages;
        bytes = stage_bytes;
    }
    __device__ __forceinline__ uint32_t parity() const { return (par >> stage) & 1u; }
    __device__ __forceinline__ void next() {
        par ^= 1u << stage;
        stage = stage + 1 == ns ? 0u : stage + 1;
    }
};

// Epoch table of a sub-group of GS periods and Es epochs (shared-memory addresses):
//   off   [Es][GS] byte offset of period g's first cell o_e(g) within strip e, whose first
//         cell is (tmin[e] & ~1) (copies start on a 16-byte boundary): u32, or u16 (W = 2)
//   tmin, tmax [Es]  smallest and largest o_e over the sub-group's present periods.
struct fold_table {
    uint32_t off, tmin, tmax;
    int Es;
    __device__ __forceinline__ int lo(int e) const { return lds_s32(tmin + 4u * (uint32_t)e); }
    __device__ __forceinline__ int hi(int e) const { return lds_s32(tmax + 4u * (uint32_t)e); }
};

__host__ __device__ constexpr int64_t table_off_bytes(int64_t Es, int GS, int W) {
    return ((Es * GS * W) + 15) & ~(int64_t)15;
}
__host__ __device__ constexpr int64_t table_bytes(int64_t Es, int GS, int W) {
    return table_off_bytes(Es, GS, W) + 8 * Es;
}

// The byte offsets of one epoch's GS periods: W = 4 bytes each, or W = 2 (two per word).
template <int GS, int W>
struct epoch_offsets {
    static constexpr int N = W == 4 ? GS : (GS + 1) / 2;
    uint32_t w[N];
    __device__ __forceinline__ void load(uint32_t a) {
        if constexpr (N >= 4) {
#pragma unroll
            for (int k = 0; k < N; k += 4)
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(w[k]), "=r"(w[k + 1]), "=r"(w[k + 2]), "=r"(w[k + 3])
                             : "r"(a + 4u * k));
        } else if constexpr (N == 2) {
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(a));
        } else if constexpr (W == 4 || GS == 2) {
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(w[0]) : "r"(a));
        } else {
            uint16_t h;
            asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(a));
            w[0] = h;
        }
    }
    __device__ __forceinline__ uint32_t operator[](int g) const {
        if constexpr (W == 4) return w[g];
        return (g & 1) ? (w[g >> 1] >> 16) : (w[g >> 1] & 0xFFFFu);
    }
};

// Bit gg set when period g0 + gg is folded at duration j: it has epochs, D_j < P (Sec. 2.3)
// and the caller's mask allows the pair.
template <int GS>
__device__ __forceinline__ unsigned period_use(const fold_smem &sm, int g0, int j) {
    const double D = sm.it.durations[j];
    const uint8_t *mask = sm.it.mask;
    unsigned use = 0u;
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        const int g = g0 + gg;
        if (sm.E[g] > 0 && D < sm.P[g] &&
            (!mask || mask[(int64_t)(sm.it.mask_k0 + g) * sm.it.J + j]))
            use |= 1u << gg;
    }
    return use;
}

__device__ __forceinline__ void record_timeout(fold_smem &sm) {
    if (!*(volatile int *)&sm.abort) {
        *(volatile int *)&sm.abort = 1;
        atomicExch(sm.it.status, CETRA_ETIMEOUT);
    }
}

// Consumers' bounded wait, called by whole warps; the result is the same for every lane
// (false if any lane's wait gave up, or if the phase is not complete and the block has
// aborted). A wait that gives up records the time-out and aborts the block.
__device__ __noinline__ bool fold_wait_slow(fold_smem &sm, uint64_t *bar, uint32_t parity) {
    bool ok = true;
    if (!mbar_test(bar, parity)) {
        ok = !*(volatile int *)&sm.abort && mbar_wait(bar, parity);
        if (!ok) record_timeout(sm);
    }
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ bool fold_wait(fold_smem &sm, uint64_t *bar, uint32_t parity) {
    if (__all_sync(0xFFFFFFFFu, mbar_test(bar, parity))) return true;  // the phase is complete
    return fold_wait_slow(sm, bar, parity);
}

// The producer's bounded wait, by its one issuing lane, which sleeps in the barrier's
// potentially blocking test instead of spinning.
__device__ __forceinline__ bool producer_wait(fold_smem &sm, uint64_t *bar, uint32_t parity) {
    if (mbar_wait(bar, parity)) return true;
    record_timeout(sm);
    return false;
}

// One bulk copy of cells [a, a + len) of grid row j into the ring's current strip.
__device__ __forceinline__ void issue_copy(fold_smem &sm, uint32_t ring0, const ring &rg, int j,
                                           int a, int len) {
    const uint32_t bytes = (uint32_t)len * (uint32_t)sizeof(float2);
    const float2 *src = sm.it.ab + (int64_t)j * sm.it.ld + a;
    fence_proxy_async();
    mbar_expect_tx(&sm.full[rg.stage], bytes);
    bulk_load_s(ring0 + rg.stage * rg.bytes, src, bytes, &sm.full[rg.stage]);
}

// A consumer thread's running maximum of each period of the sub-group, in shared memory: slot
// gg of thread c at [gg * FT_THREADS + c], the largest 2 LR so far and the flat index of its
// window. They are read once per tile and written only when a maximum changes, so they take
// no registers in the hot loop.
struct best_slots {
    float *lr2;
    uint32_t *at;
};

template <int GS>
__device__ __forceinline__ void init_best(best_slots bs) {
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        bs.lr2[gg * FT_THREADS + threadIdx.x] = -1.0f;
        bs.at[gg * FT_THREADS + threadIdx.x] = 0u;
    }
}

// Per-thread best of each period (the largest 2 LR, first in (j, i) order on ties) -> the
// slot's best key in shared memory.
template <int GS>
__device__ __forceinline__ void publish_best(fold_smem &sm, int g0, best_slots bs) {
    const int c = threadIdx.x;
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        const float b = bs.lr2[gg * FT_THREADS + c];
        unsigned long long key = b >= 0.0f ? make_key(0.5f * b, bs.at[gg * FT_THREADS + c]) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, key, o);
            key = u > key ? u : key;
        }
        if ((threadIdx.x & 31) == 0 && key) atomicMax(&sm.best[g0 + gg], key);
    }
}

// Exact running maximum over one window sum (x, y) = (sum A, sum B) at flat index at:
// 2 LR = x * (x / y); a null sum gives NaN, never a maximum; the first of equal values stays.
__device__ __forceinline__ void take_max(float x, float y, uint32_t at, best_slots bs, int gg) {
    const int k = gg * FT_THREADS + threadIdx.x;
    const float lr2 = x * __fdividef(x, y);
    if (lr2 > bs.lr2[k]) {
        bs.lr2[k] = lr2;
        bs.at[k] = at;
    }
}

// ---------------------------------------------------------------------------------------------
// Main path: tiles of T = FT_THREADS R phases, one strip per epoch.

// Live epochs of a tile starting at phase i0: e < Es with tmin[e] < I - i0 (tmin is
// nondecreasing in e, so they are a prefix); nE only shrinks as i0 grows.
__device__ __forceinline__ int live_epochs(const fold_table &tb, int nE, int I, int i0) {
    while (nE > 0 && tb.lo(nE - 1) >= I - i0) --nE;
    return nE;
}

// Rows of a tile whose row has `rem` phases left (rem >= 1): the last tile of a row folds
// only the rows of FT_THREADS phases that hold some phase of the sub-group, so its lanes past
// the last phase neither copy nor load cells. (Sub-groups of fewer than 4 periods, which only
// tables too large for 4 give, always fold R rows: fewer kernel variants.)
template <int GS, int R>
__device__ __forceinline__ int tile_rows(int rem) {
    if constexpr (GS < 4 || R == 1) {
        return R;
    } else {
        const int rows = (rem + FT_THREADS - 1) / FT_THREADS;
        return rows < R ? rows : R;
    }
}

// Run by the producer warp's first lane alone.
template <int GS, int R>
__device__ void produce_main(fold_smem &sm, uint32_t ring0, const fold_table &tb, int g0,
                             int nph_sub, ring &rg) {
    constexpr int T = FT_THREADS * R;
    const int I = sm.it.I;
    for (int j = sm.it.jlo; j < sm.it.jhi; ++j) {
        if (!period_use<GS>(sm, g0, j)) continue;
        int nE = tb.Es;
        for (int i0 = 0; i0 < nph_sub; i0 += T) {
            nE = live_epochs(tb, nE, I, i0);
            const int TL = FT_THREADS * tile_rows<GS, R>(nph_sub - i0);  // phases of this tile
            for (int e = 0; e < nE; ++e) {
                if (!producer_wait(sm, &sm.empty[rg.stage], rg.parity() ^ 1u)) return;
                const int a = i0 + (tb.lo(e) & ~1);
                issue_copy(sm, ring0, rg, j, a, ((i0 + tb.hi(e) + TL - a) + 1) & ~1);
                rg.next();
            }
        }
    }
}

// Epochs 2 .. nE-1 of a tile (epochs 0 and 1 started the sums): ALL = every period of the
// sub-group is folded at this duration (no per-period test in the loop).
template <int GS, int R, int W, bool KAHAN, bool ALL>
__device__ __forceinline__ bool consume_epochs(fold_smem &sm, const fold_table &tb, int nE,
                                               unsigned use, uint32_t mine, uint64_t (&acc)[GS][R],
                                               uint64_t (&cmp)[KAHAN ? GS : 1][KAHAN ? R : 1],
                                               ring &rg) {
    int e = 2;
    if constexpr (KAHAN) {
        // The compensated form takes the epochs in groups of FT_KAHAN_GROUP (when the ring has
        // that many stages): the group's cells are added plainly, and the group sum enters the
        // compensated sum, so a cell costs 1 + 4 / FT_KAHAN_GROUP packed operations instead of
        // 5 and the shared-memory loads stay the bound. Error: FT_KAHAN_GROUP - 1 roundings
        // per group sum on top of the compensated sum's own bound.
        constexpr int KG = FT_KAHAN_GROUP;
        if (rg.ns >= (uint32_t)KG) {
            for (; e + KG - 1 < nE; e += KG) {
                uint32_t st[KG], ad[KG];
#pragma unroll
                for (int k = 0; k < KG; ++k) {
                    if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return false;
                    st[k] = rg.stage;
                    ad[k] = mine + rg.stage * rg.bytes;
                    rg.next();
                }
                epoch_offsets<GS, W> off[KG];
#pragma unroll
                for (int k = 0; k < KG; ++k) off[k].load(tb.off + (uint32_t)((e + k) * GS * W));
#pragma unroll
                for (int gg = 0; gg < GS; ++gg) {
                    if (!ALL && !((use >> gg) & 1u)) continue;
                    uint64_t v[KG][R];
#pragma unroll
                    for (int k = 0; k < KG; ++k) lds_rows<0, R>(v[k], ad[k] + off[k][gg]);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        uint64_t g = v[0][r];
#pragma unroll
                        for (int k = 1; k < KG; ++k) g = sum_pair(g, v[k][r]);
                        kahan_add_pair(acc[gg][r], cmp[gg][r], g);
                    }
                }
#pragma unroll
                for (int k = 0; k < KG; ++k) mbar_arrive(&sm.empty[st[k]]);
            }
        }
    }
    for (; e < nE; ++e) {
        if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return false;
        const uint32_t a = mine + rg.stage * rg.bytes;
        epoch_offsets<GS, W> off;
        off.load(tb.off + (uint32_t)(e * GS * W));
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            if (!ALL && !((use >> gg) & 1u)) continue;
            const uint32_t ag = a + off[gg];
            uint64_t v[R];
            lds_rows<0, R>(v, ag);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (KAHAN)
                    kahan_add_pair(acc[gg][r], cmp[gg][r], v[r]);
                else
                    add_pair(acc[gg][r], v[r]);
            }
        }
        mbar_arrive(&sm.empty[rg.stage]);
        rg.next();
    }
    return true;
}

// One tile of the main path: epochs 0 .. nE-1 into acc, then the running maxima. SHORT: the
// tile has at most 3 live epochs and runs as straight-line code (no loop-carried sums).
template <int GS, int R, int W, bool KAHAN, bool SHORT>
__device__ __forceinline__ bool consume_tile(fold_smem &sm, const fold_table &tb, int g0, int j,
                                             int i0, int nE, unsigned use, bool all_used,
                                             int nmin, uint32_t mine, best_slots bs, ring &rg) {
    constexpr int T = FT_THREADS * R;
    const int c = threadIdx.x;
    uint64_t acc[GS][R];
    uint64_t cmp[KAHAN ? GS : 1][KAHAN ? R : 1];  // minus the Kahan compensation
    // Epoch 0: every period's cell is its phase cell (o_0 = 0), one load for all. Epoch 1 then
    // starts each sum as (epoch-0 cell + epoch-1 cell).
    if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return false;
    uint64_t v0[R];
    {
        const uint32_t a = mine + rg.stage * rg.bytes;
        lds_rows<0, R>(v0, a);
        mbar_arrive(&sm.empty[rg.stage]);
    }
    rg.next();
    if (KAHAN || nE < 2) {
#pragma unroll
        for (int gg = 0; gg < GS; ++gg)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[gg][r] = v0[r];
        if constexpr (KAHAN) {
#pragma unroll
            for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                for (int r = 0; r < R; ++r) cmp[gg][r] = 0ull;
        }
    }
    if (nE >= 2) {
        if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return false;
        const uint32_t a = mine + rg.stage * rg.bytes;
        epoch_offsets<GS, W> off;
        off.load(tb.off + (uint32_t)(GS * W));
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            const uint32_t ag = a + off[gg];
            uint64_t v[R];
            lds_rows<0, R>(v, ag);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (KAHAN)
                    kahan_add_pair(acc[gg][r], cmp[gg][r], v[r]);
                else
                    acc[gg][r] = sum_pair(v0[r], v[r]);
            }
        }
        mbar_arrive(&sm.empty[rg.stage]);
        rg.next();
    }
    if constexpr (SHORT) {
        if (nE >= 3) {
            if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return false;
            const uint32_t a = mine + rg.stage * rg.bytes;
            epoch_offsets<GS, W> off;
            off.load(tb.off + (uint32_t)(2 * GS * W));
#pragma unroll
            for (int gg = 0; gg < GS; ++gg) {
                const uint32_t ag = a + off[gg];
                uint64_t v[R];
                lds_rows<0, R>(v, ag);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if constexpr (KAHAN)
                        kahan_add_pair(acc[gg][r], cmp[gg][r], v[r]);
                    else
                        add_pair(acc[gg][r], v[r]);
                }
            }
            mbar_arrive(&sm.empty[rg.stage]);
            rg.next();
        }
    } else {
        const bool ok =
            all_used ? consume_epochs<GS, R, W, KAHAN, true>(sm, tb, nE, use, mine, acc, cmp, rg)
                     : consume_epochs<GS, R, W, KAHAN, false>(sm, tb, nE, use, mine, acc, cmp, rg);
        if (!ok) return false;
    }
    // 2 LR = SA^2 / SB per (period, phase); the running maximum keeps the first (smallest j,
    // then smallest i) of equal values. Whole tiles (nmin: the phases every used period has)
    // first run the candidate test over all their windows.
    float m = i0 + T > nmin ? 1.0f : -1.0f;  // a ragged tile takes the exact comparisons
#pragma unroll
    for (int gg = 0; gg < GS; ++gg) {
        if (!all_used && !((use >> gg) & 1u)) continue;
        const float h = bs.lr2[gg * FT_THREADS + c] * kCandidate;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t v = acc[gg][r];
            if constexpr (KAHAN) add_pair(v, cmp[gg][r]);
            float x, y;
            split_pair(v, x, y);
            m = fmaxf(m, fmaf(x, x, -(h * y)));
        }
    }
    if (m > 0.0f) {
        const uint32_t jI = (uint32_t)j * (uint32_t)sm.it.I;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            if (!((use >> gg) & 1u)) continue;
            const int nph = sm.nph[g0 + gg];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = i0 + c + r * FT_THREADS;
                uint64_t v = acc[gg][r];
                if constexpr (KAHAN) add_pair(v, cmp[gg][r]);
                float x, y;
                split_pair(v, x, y);
                if (i < nph)
                    take_max(x, y, jI + (uint32_t)i, bs, gg);
            }
        }
    }
    return true;
}

// A tile of `rows` rows (rows <= RL): the variant with exactly that many, straight-line when
// it has at most 3 live epochs.
template <int GS, int R, int W, bool KAHAN, int RL>
__device__ __forceinline__ bool consume_tile_rows(int rows, fold_smem &sm, const fold_table &tb,
                                                  int g0, int j, int i0, int nE, unsigned use,
                                                  bool all_used, int nmin, uint32_t mine,
                                                  best_slots bs, ring &rg) {
    if constexpr (RL > 1 && GS >= 4) {
        if (rows < RL)
            return consume_tile_rows<GS, R, W, KAHAN, RL - 1>(rows, sm, tb, g0, j, i0, nE, use,
                                                              all_used, nmin, mine, bs, rg);
    }
    return nE <= 3 ? consume_tile<GS, RL, W, KAHAN, true>(sm, tb, g0, j, i0, nE, use, all_used,
                                                          nmin, mine, bs, rg)
                   : consume_tile<GS, RL, W, KAHAN, false>(sm, tb, g0, j, i0, nE, use, all_used,
                                                           nmin, mine, bs, rg);
}

template <int GS, int R, int W, bool KAHAN>
__device__ void consume_main(fold_smem &sm, uint32_t ring0, best_slots bs, const fold_table &tb,
                             int g0, int nph_sub, ring &rg) {
    constexpr int T = FT_THREADS * R;
    const int c = threadIdx.x;
    const uint32_t mine = ring0 + (uint32_t)c * (uint32_t)sizeof(float2);
    init_best<GS>(bs);
    for (int j = sm.it.jlo; j < sm.it.jhi; ++j) {
        const unsigned use = period_use<GS>(sm, g0, j);
        if (!use) continue;
        const bool all_used = use == (1u << GS) - 1u;
        int nmin = nph_sub;  // phases every used period has
#pragma unroll
        for (int gg = 0; gg < GS; ++gg)
            if ((use >> gg) & 1u) nmin = min(nmin, sm.nph[g0 + gg]);
        int nE = tb.Es;
        for (int i0 = 0; i0 < nph_sub; i0 += T) {
            nE = live_epochs(tb, nE, sm.it.I, i0);
            // (a wait that gave up ends the path at once: the main path has no block barrier,
            // so every thread still meets the caller's next one)
            const bool ok = consume_tile_rows<GS, R, W, KAHAN, R>(
                tile_rows<GS, R>(nph_sub - i0), sm, tb, g0, j, i0, nE, use, all_used, nmin, mine,
                bs, rg);
            if (!ok) return;
        }
    }
    publish_best<GS>(sm, g0, bs);
}

// ---------------------------------------------------------------------------------------------
// Epoch-sliced path: a sub-group whose periods all have few phases (nph <= Tp <= T/2,
// Tp = max(32, nph)). The lanes L = c + FT_THREADS r form H = floor(T / Tp) slices of Tp
// phases (lane L: slice L / Tp, phase L % Tp; lanes past H Tp idle); slice h folds epochs
// e = s H + h of super-epoch s, one strip per super-epoch. The H partial sums of a phase are
// then added in slice order through shared memory. (Strip bound: tmin grows by at most Tp
// per epoch, since o_{e+1} - o_e <= ceil(Ps) <= Tp for the period that attains tmin[e], so a
// super-epoch needs at most H Tp + spread + 3 <= T + spread + 3 cells; the table check keeps
// spread <= FT_STRIP - T - 8 for this path.)

__device__ __forceinline__ bool live_epoch(const fold_table &tb, int e, int I) {
    return e < tb.Es && tb.lo(e) < I;
}

template <int GS, int R>
__device__ void produce_sliced(fold_smem &sm, uint32_t ring0, const fold_table &tb, int g0,
                               int Tp, ring &rg) {
    constexpr int T = FT_THREADS * R;
    const int H = T / Tp;
    const int I = sm.it.I;
    const bool leader = (threadIdx.x & 31) == 0;
    for (int j = sm.it.jlo; j < sm.it.jhi; ++j) {
        const unsigned use = period_use<GS>(sm, g0, j);
        if (!use) continue;
        for (int s = 0; live_epoch(tb, s * H, I); ++s) {
            // (after an abort this only keeps the loop, and the barriers below, in step)
            if (leader && producer_wait(sm, &sm.empty[rg.stage], rg.parity() ^ 1u)) {
                const int e0 = s * H;
                const int a = tb.lo(e0) & ~1;
                int end = 0;
                for (int h = 0; h < H; ++h)
                    if (live_epoch(tb, e0 + h, I)) end = max(end, tb.hi(e0 + h) + Tp);
                issue_copy(sm, ring0, rg, j, a, ((end - a) + 1) & ~1);
            }
            __syncwarp();
            rg.next();
        }
        // the consumers' slice reduction: two block barriers per folded period
        for (int gg = 0; gg < GS; ++gg)
            if ((use >> gg) & 1u) {
                block_sync();
                block_sync();
            }
    }
}

template <int GS, int R, int W, bool KAHAN>
__device__ void consume_sliced(fold_smem &sm, uint32_t ring0, uint64_t *part, best_slots bs,
                               const fold_table &tb, int g0, int Tp, ring &rg) {
    constexpr int T = FT_THREADS * R;
    const int H = T / Tp;
    const int c = threadIdx.x;
    const int I = sm.it.I;
    int slice[R], phase[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int L = c + r * FT_THREADS;
        slice[r] = L / Tp;
        phase[r] = L - slice[r] * Tp;
    }
    init_best<GS>(bs);
    for (int j = sm.it.jlo; j < sm.it.jhi; ++j) {
        const unsigned use = period_use<GS>(sm, g0, j);
        if (!use) continue;
        const bool all_used = use == (1u << GS) - 1u;
        uint64_t acc[GS][R];
        uint64_t cmp[KAHAN ? GS : 1][KAHAN ? R : 1];
#pragma unroll
        for (int gg = 0; gg < GS; ++gg)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[gg][r] = 0ull;
        if constexpr (KAHAN) {
#pragma unroll
            for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                for (int r = 0; r < R; ++r) cmp[gg][r] = 0ull;
        }
        for (int s = 0; live_epoch(tb, s * H, I); ++s) {
            // after an abort the loop runs on without work, to keep the barriers below in step
            if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) {
                rg.next();
                continue;
            }
            const int a_s = tb.lo(s * H) & ~1;
            const uint32_t stage = ring0 + rg.stage * rg.bytes;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (slice[r] >= H) continue;  // lane past the last whole slice
                const int e = s * H + slice[r];
                if (!live_epoch(tb, e, I)) continue;
                const uint32_t lb =
                    stage + (uint32_t)(phase[r] + (tb.lo(e) & ~1) - a_s) * (uint32_t)sizeof(float2);
                epoch_offsets<GS, W> off;
                off.load(tb.off + (uint32_t)(e * GS * W));
#pragma unroll
                for (int gg = 0; gg < GS; ++gg) {
                    if (!all_used && !((use >> gg) & 1u)) continue;
                    const uint64_t v = lds_pair(lb + off[gg]);
                    if constexpr (KAHAN)
                        kahan_add_pair(acc[gg][r], cmp[gg][r], v);
                    else
                        add_pair(acc[gg][r], v);
                }
            }
            mbar_arrive(&sm.empty[rg.stage]);
            rg.next();
        }
        // the slices' partial sums of each phase, added in slice order
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            if (!((use >> gg) & 1u)) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                uint64_t v = acc[gg][r];
                if constexpr (KAHAN) add_pair(v, cmp[gg][r]);
                part[c + r * FT_THREADS] = v;
            }
            block_sync();
            const int nph = sm.nph[g0 + gg];
            for (int phi = c; phi < Tp; phi += FT_THREADS) {
                uint64_t v = part[phi];
                for (int h = 1; h < H; ++h) add_pair(v, part[h * Tp + phi]);
                float x, y;
                split_pair(v, x, y);
                if (phi < nph && y > 0.0f)
                    take_max(x, y, (uint32_t)j * (uint32_t)I + (uint32_t)phi, bs, gg);
            }
            block_sync();
        }
    }
    publish_best<GS>(sm, g0, bs);
}

// ---------------------------------------------------------------------------------------------
// Duration-packed path: a sub-group of 4 or 8 periods with few phases (Tp = nph rounded up to
// even, Tp <= T/2) in a work item of several durations. The lanes L = c + FT_THREADS r form
// H = T / Tp rows of Tp phases (lane L: row L / Tp, phase L % Tp; lanes past H Tp idle), and
// row h of a tile is the h-th duration of the sub-group's list (the durations at which any of
// its periods is folded), so a tile folds H durations at once. Every lane reads the same epoch
// at the same time: the producer copies, for each epoch, one segment of cells
// [lo_e & ~1, hi_e + Tp] per row into that row's part of the strip (segments `seg` cells apart,
// seg = Tp mod 32, so a warp that spans two rows reads as if they were contiguous: no bank
// conflicts), each lane folds every epoch of its own (duration, phase) window sums, and no
// partial sums meet through shared memory. (The epoch-sliced path instead splits one duration
// row's epochs over the lanes and adds the slices through shared memory behind two block
// barriers per folded period; it stays for work items of one duration.)

// The sub-group's durations in [jlo, jhi) (jhi - jlo <= FT_PACK_MAXJ) at which some period is
// folded, in ascending order with their period_use bits (the producer warp, 32 at a time).
template <int GS>
__device__ void build_pack_list(fold_smem &sm, int g0) {
    const int lane = threadIdx.x & 31;
    int n = 0;
    for (int jb = sm.it.jlo; jb < sm.it.jhi; jb += 32) {
        const int j = jb + lane;
        const unsigned u = j < sm.it.jhi ? period_use<GS>(sm, g0, j) : 0u;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, u != 0u);
        if (u) {
            const int k = n + __popc(bal & ((1u << lane) - 1u));
            sm.pack_j[k] = (int16_t)j;
            sm.pack_use[k] = (uint8_t)u;
        }
        n += __popc(bal);
    }
    if (lane == 0) sm.pack_n = n;
}

// Run by the producer warp's first lane alone: per tile of H listed durations and per live
// epoch, one strip of H segments (one bulk copy per row, one barrier arrival for all).
__device__ void produce_packed(fold_smem &sm, uint32_t ring0, const fold_table &tb, int Tp, int H,
                               int seg, ring &rg) {
    const int nJ = sm.pack_n;
    const int nE = live_epochs(tb, tb.Es, sm.it.I, 0);
    const uint32_t seg_bytes = (uint32_t)seg * (uint32_t)sizeof(float2);
    for (int t0 = 0; t0 < nJ; t0 += H) {
        const int nr = min(H, nJ - t0);
        for (int e = 0; e < nE; ++e) {
            if (!producer_wait(sm, &sm.empty[rg.stage], rg.parity() ^ 1u)) return;
            const int a = tb.lo(e) & ~1;
            const uint32_t bytes = (uint32_t)(((tb.hi(e) + Tp - a) + 1) & ~1) * (uint32_t)sizeof(float2);
            const uint32_t dst = ring0 + rg.stage * rg.bytes;
            fence_proxy_async();
            mbar_expect_tx(&sm.full[rg.stage], bytes * (uint32_t)nr);
            for (int h = 0; h < nr; ++h) {
                const float2 *src = sm.it.ab + (int64_t)sm.pack_j[t0 + h] * sm.it.ld + a;
                bulk_load_s(dst + (uint32_t)h * seg_bytes, src, bytes, &sm.full[rg.stage]);
            }
            rg.next();
        }
    }
}

template <int GS, int R, int W, bool KAHAN>
__device__ void consume_packed(fold_smem &sm, uint32_t ring0, best_slots bs, const fold_table &tb,
                               int g0, int Tp, int H, int seg, ring &rg) {
    const int c = threadIdx.x;
    const int nJ = sm.pack_n;
    const uint32_t I = (uint32_t)sm.it.I;
    const int nE = live_epochs(tb, tb.Es, sm.it.I, 0);
    int row[R], ph[R];
    uint32_t base[R];  // the lane's cell in its row's segment (bytes from the strip's start)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int L = c + r * FT_THREADS;
        row[r] = L / Tp;
        ph[r] = L - row[r] * Tp;
        base[r] = row[r] < H ? ((uint32_t)row[r] * (uint32_t)seg + (uint32_t)ph[r]) *
                                   (uint32_t)sizeof(float2)
                             : 0u;  // idle lane: reads row 0, never used
    }
    init_best<GS>(bs);
    for (int t0 = 0; t0 < nJ; t0 += H) {
        const int nr = min(H, nJ - t0);
        uint64_t acc[GS][R];
        uint64_t cmp[KAHAN ? GS : 1][KAHAN ? R : 1];
        // epoch 0: every period's cell is its phase cell (o_0 = 0), one load for all
        if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return;
        {
            const uint32_t a = ring0 + rg.stage * rg.bytes;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint64_t v = lds_pair(a + base[r]);
#pragma unroll
                for (int gg = 0; gg < GS; ++gg) acc[gg][r] = v;
            }
            mbar_arrive(&sm.empty[rg.stage]);
        }
        rg.next();
        if constexpr (KAHAN) {
#pragma unroll
            for (int gg = 0; gg < GS; ++gg)
#pragma unroll
                for (int r = 0; r < R; ++r) cmp[gg][r] = 0ull;
        }
        for (int e = 1; e < nE; ++e) {
            if (!fold_wait(sm, &sm.full[rg.stage], rg.parity())) return;
            const uint32_t a = ring0 + rg.stage * rg.bytes;
            epoch_offsets<GS, W> off;
            off.load(tb.off + (uint32_t)(e * GS * W));
            uint32_t ar[R];
#pragma unroll
            for (int r = 0; r < R; ++r) ar[r] = a + base[r];
#pragma unroll
            for (int gg = 0; gg < GS; ++gg) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint64_t v = lds_pair(ar[r] + off[gg]);
                    if constexpr (KAHAN)
                        kahan_add_pair(acc[gg][r], cmp[gg][r], v);
                    else
                        add_pair(acc[gg][r], v);
                }
            }
            mbar_arrive(&sm.empty[rg.stage]);
            rg.next();
        }
        // running maxima, in (duration, phase) order within the thread
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (row[r] >= nr) continue;
            const int k = t0 + row[r];
            const uint32_t at = (uint32_t)sm.pack_j[k] * I + (uint32_t)ph[r];
            const unsigned u = sm.pack_use[k];
#pragma unroll
            for (int gg = 0; gg < GS; ++gg) {
                if (!((u >> gg) & 1u) || ph[r] >= sm.nph[g0 + gg]) continue;
                uint64_t v = acc[gg][r];
                if constexpr (KAHAN) add_pair(v, cmp[gg][r]);
                float x, y;
                split_pair(v, x, y);
                take_max(x, y, at, bs, gg);
            }
        }
    }
    publish_best<GS>(sm, g0, bs);
}

// ---------------------------------------------------------------------------------------------
// One period whose epoch table does not fit: straight from global memory (consumers only).
__device__ void fold_direct(fold_smem &sm, int g) {
    const int c = threadIdx.x;
    const double Ps = sm.Ps[g];
    const int I = sm.it.I;
    unsigned long long best = 0ull;
    for (int j = sm.it.jlo; j < sm.it.jhi; ++j) {
        if (!period_use<1>(sm, g, j)) continue;
        const float2 *row = sm.it.ab + (int64_t)j * sm.it.ld;
        for (int i = c; i < sm.nph[g]; i += FT_THREADS) {
            float2 acc = make_float2(0.f, 0.f);
            for (int64_t e = 0;; ++e) {
                const int64_t cell = i + epoch_offset(e, Ps);
                if (cell >= I) break;
                add2(acc, row[cell]);
            }
            if (acc.y > 0.0f) {
                const float lr = 0.5f * (acc.x * __fdividef(acc.x, acc.y));
                const unsigned long long key = make_key(lr, (uint32_t)j * (uint32_t)I + (uint32_t)i);
                if (key > best) best = key;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = u > best ? u : best;
    }
    if ((c & 31) == 0 && best) atomicMax(&sm.best[g], best);
}

// ---------------------------------------------------------------------------------------------

// Slot t of a group (thread t < FT_G): P, Ps = P/s in t0 steps, the number of phases and an
// upper bound on the epochs with o_e < I.
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
    sm.best[t] = 0ull;
}

// Build the epoch table of sub-group [g0, g0 + GS) (all threads), offsets W bytes wide. Sets
// sm.bad when some epoch's spread leaves no room for a tile in a strip, sm.tight when it
// leaves less than the sliced path's margin, sm.spread to the widest spread. Offsets beyond
// the t0 grid are kept (their cells are the zero padding after each grid row), so a strip
// never needs clipping.
template <int GS, int W>
__device__ void build_table(fold_smem &sm, unsigned char *raw, int g0, int Es, int T) {
    unsigned char *off = raw;
    int32_t *tmin = reinterpret_cast<int32_t *>(raw + table_off_bytes(Es, GS, W));
    int32_t *tmax = tmin + Es;
    bool bad = false, tight = false;
    int64_t widest = 0;
    for (int e = threadIdx.x; e < Es; e += blockDim.x) {
        int64_t o[GS];
        int64_t mn = INT64_MAX, mx = INT64_MIN;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            const int g = g0 + gg;
            o[gg] = -1;
            if (sm.E[g] > 0) {
                int64_t v = epoch_offset(e, sm.Ps[g]);
                v = v < (int64_t)1 << 30 ? v : (int64_t)1 << 30;
                o[gg] = v;
                mn = v < mn ? v : mn;
                mx = v > mx ? v : mx;
            }
        }
        const int64_t base = mn & ~(int64_t)1;
        const int64_t spread = mx - mn;
        if (spread > FT_STRIP - T - 2) bad = true;
        if (spread > FT_STRIP - T - 8) tight = true;
        widest = spread > widest ? spread : widest;
#pragma unroll
        for (int gg = 0; gg < GS; ++gg) {
            int64_t d = o[gg] >= 0 ? (o[gg] - base) * (int64_t)sizeof(float2) : 0;
            d = d >= 0 && d < 65536 ? d : 0;
            if constexpr (W == 4)
                reinterpret_cast<uint32_t *>(off)[e * GS + gg] = (uint32_t)d;
            else
                reinterpret_cast<uint16_t *>(off)[e * GS + gg] = (uint16_t)d;
        }
        tmin[e] = (int32_t)mn;
        tmax[e] = (int32_t)mx;
    }
    if (bad) sm.bad = 1;
    if (tight) sm.tight = 1;
    if (!bad && widest > 0) atomicMax(&sm.spread, (int)widest);
}

template <int GS>
__device__ __forceinline__ void build_table_w(fold_smem &sm, unsigned char *raw, int g0, int Es,
                                              int T, int W) {
    if (W == 4)
        build_table<GS, 4>(sm, raw, g0, Es, T);
    else
        build_table<GS, 2>(sm, raw, g0, Es, T);
}

template <int GS, int R, int W, bool KAHAN>
__device__ void fold_subgroup(fold_smem &sm, uint32_t ring0, const fold_table &tb, uint64_t *part,
                              best_slots bs, bool sliced, int Tp, int g0, int nph_sub, int H,
                              int seg, ring &rg) {
    const bool producer = threadIdx.x >= FT_THREADS;
    if (H > 0) {
        // duration-packed (no block barrier, as the main path)
        if constexpr (GS >= 4) {
            if (producer) {
                if ((threadIdx.x & 31) == 0) produce_packed(sm, ring0, tb, Tp, H, seg, rg);
                __syncwarp();
            } else {
                consume_packed<GS, R, W, KAHAN>(sm, ring0, bs, tb, g0, Tp, H, seg, rg);
            }
        }
    } else if (sliced) {
        if (producer)
            produce_sliced<GS, R>(sm, ring0, tb, g0, Tp, rg);
        else
            consume_sliced<GS, R, W, KAHAN>(sm, ring0, part, bs, tb, g0, Tp, rg);
    } else if (producer) {
        // the main path has no block barrier: the producer's first lane runs it alone
        if ((threadIdx.x & 31) == 0) produce_main<GS, R>(sm, ring0, tb, g0, nph_sub, rg);
        __syncwarp();
    } else {
        consume_main<GS, R, W, KAHAN>(sm, ring0, bs, tb, g0, nph_sub, rg);
    }
}

template <int GS, int R, bool KAHAN>
__device__ __forceinline__ void fold_subgroup_w(fold_smem &sm, uint32_t ring0,
                                                const fold_table &tb, uint64_t *part,
                                                best_slots bs, bool sliced, int Tp, int g0,
                                                int nph_sub, int H, int seg, ring &rg, int W) {
    if (W == 4)
        fold_subgroup<GS, R, 4, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                       rg);
    else
        fold_subgroup<GS, R, 2, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                       rg);
}

// Fold the group whose slot metadata and work item are in `sm` (all threads): every sub-group
// (8 -> 4 -> 2 -> 1 periods, as the table allows) in turn; slot g's best key ends in
// sm.best[g]. A wait that gave up leaves sm.abort set.
template <bool KAHAN, int R>
__device__ __forceinline__ void fold_group(fold_smem &sm, unsigned char *raw, unsigned char *tab, best_slots bs,
                           ring &rg) {
    constexpr int T = FT_THREADS * R;
    for (int g0 = 0; g0 < FT_G;) {
        int GS = sm.it.gmax;
        while (g0 % GS) GS >>= 1;
        int Es = 0, W = 4;
        bool table_ok = false;
        for (;;) {
            Es = 0;
            for (int g = g0; g < g0 + GS; ++g) Es = max(Es, sm.E[g]);
            if (Es == 0) break;  // no period of the sub-group has a phase
            // 32-bit offsets when they fit, else 16-bit
            W = table_bytes(Es, GS, 4) <= FT_TAB_BYTES ? 4 : 2;
            if (table_bytes(Es, GS, W) > FT_TAB_BYTES) {
                if (GS > 1) {
                    GS >>= 1;
                    continue;
                }
                break;  // a single period with too many epochs: no table
            }
            block_sync();  // everyone is done with the previous table
            if (threadIdx.x == 0) sm.bad = sm.tight = sm.spread = 0;
            block_sync();
            if (GS == 8)
                build_table_w<8>(sm, tab, g0, Es, T, W);
            else if (GS == 4)
                build_table_w<4>(sm, tab, g0, Es, T, W);
            else if (GS == 2)
                build_table_w<2>(sm, tab, g0, Es, T, W);
            else
                build_table_w<1>(sm, tab, g0, Es, T, W);
            block_sync();
            if (sm.bad && GS > 1) {
                GS >>= 1;
                continue;
            }
            table_ok = !sm.bad;
            break;
        }
        int nph_sub = 0;
        for (int g = g0; g < g0 + GS; ++g) nph_sub = max(nph_sub, sm.nph[g]);
        if (Es == 0 || nph_sub == 0) {
            g0 += GS;
            continue;
        }
        if (!table_ok) {
            // GS == 1 here
            if (threadIdx.x < FT_THREADS) fold_direct(sm, g0);
            g0 += GS;
            continue;
        }
        fold_table tb;
        tb.off = smem_u32(tab);
        tb.tmin = tb.off + (uint32_t)table_off_bytes(Es, GS, W);
        tb.tmax = tb.tmin + 4u * (uint32_t)Es;
        tb.Es = Es;
        int Tp = max(32, nph_sub);  // phases per epoch slice
        const bool sliced = !sm.tight && 2 * Tp <= T;
        // strips as long as this sub-group's copies can be (a tile plus the widest spread,
        // rounded to whole 16-byte units), as many as the ring holds (at least 3); the sliced
        // path keeps the last one for the slices' partial sums (T pairs <= one strip)
        uint32_t stage_bytes = (uint32_t)((T + sm.spread + 5) & ~1) * (uint32_t)sizeof(float2);
        // The duration-packed path takes a short-period sub-group of 4 or 8 periods when its
        // work item has several durations and at least half of its tiles' lanes have work:
        // rows of Tp = nph rounded up to even phases, H = T / Tp rows per tile, segments of
        // seg = Tp mod 32 cells (>= Tp + spread + 3), at least two strips in the ring.
        int H = 0, seg = 0;
        if (sliced && GS >= 4 && sm.it.jhi - sm.it.jlo >= 2 &&
            sm.it.jhi - sm.it.jlo <= FT_PACK_MAXJ) {
            if (threadIdx.x >= FT_THREADS) {
                if (GS == 8)
                    build_pack_list<8>(sm, g0);
                else
                    build_pack_list<4>(sm, g0);
            }
            block_sync();
            const int nJ = sm.pack_n;
            const int Tq = (nph_sub + 1) & ~1;
            const int sq = Tq + 32 * ((sm.spread + 3 + 31) / 32);
            int Hq = min(T / Tq, nJ);
            Hq = min(Hq, (int)(FT_RING_BYTES / (2u * (uint32_t)sq * (uint32_t)sizeof(float2))));
            const int tiles = Hq > 0 ? (nJ + Hq - 1) / Hq : 0;
            if (Hq >= 2 && 2 * nJ * Tq >= tiles * T) {
                H = Hq;
                seg = sq;
                Tp = Tq;
                stage_bytes = (uint32_t)(H * seg) * (uint32_t)sizeof(float2);
            }
        }
        const uint32_t ns = min((uint32_t)FT_NSTAGE, (uint32_t)FT_RING_BYTES / stage_bytes);
        rg.start(sliced && H == 0 ? ns - 1 : ns, stage_bytes);
        uint64_t *part = reinterpret_cast<uint64_t *>(raw + (ns - 1) * stage_bytes);
        const uint32_t ring0 = smem_u32(raw);
        if (GS == 8)
            fold_subgroup_w<8, R, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                         rg, W);
        else if (GS == 4)
            fold_subgroup_w<4, R, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                         rg, W);
        else if (GS == 2)
            fold_subgroup_w<2, R, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                         rg, W);
        else
            fold_subgroup_w<1, R, KAHAN>(sm, ring0, tb, part, bs, sliced, Tp, g0, nph_sub, H, seg,
                                         rg, W);
        g0 += GS;
    }
}

// Block start: barriers (the full ones expect the producer's one arrival, the empty ones one
// arrival per consumer thread).
__device__ __forceinline__ void fold_init_barriers(fold_smem &sm) {
    if (threadIdx.x == 0) {
        for (int st = 0; st < FT_NSTAGE; ++st) {
            mbar_init(&sm.full[st], 1);
            mbar_init(&sm.empty[st], FT_THREADS);
        }
        fence_mbar_init();
        sm.abort = 0;
    }
}

// A block that aborted: the producer's first lane waits (bounded) for the last fill of every
// strip to land, so that no copy lands in shared memory after the block exits. (A strip
// never filled has parity bit 0: its wait on phase parity 1 passes at once.)
__device__ void drain_copies(fold_smem &sm, const ring &rg) {
    if (threadIdx.x != FT_THREADS) return;  // the producer's issuing lane holds the ring state
    for (int s = 0; s < FT_NSTAGE; ++s) mbar_wait(&sm.full[s], ((rg.par >> s) & 1u) ^ 1u);
}

// Dynamic shared memory: the strip ring, the epoch table, the consumers' running maxima.
__device__ __forceinline__ void fold_smem_views(unsigned char *raw, unsigned char *&tab,
                                                best_slots &bs) {
    tab = raw + FT_RING_BYTES;
    bs.lr2 = reinterpret_cast<float *>(tab + FT_TAB_BYTES);
    bs.at = reinterpret_cast<uint32_t *>(bs.lr2 + FT_G * FT_THREADS);
}

}  // namespace
