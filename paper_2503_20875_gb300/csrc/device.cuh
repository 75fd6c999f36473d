// Device helpers shared by the kernel translation units (kernels.cu, fold.cu): packed FP32x2
// arithmetic, the FP64 index arithmetic of the paper's nearest-neighbour rules, the per-period
// key, shared-memory barriers and 1-D bulk copies. Every function is internal to the library.
#pragma once

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

// Per-period key: larger LR wins; on equal LR the smaller flat index j*I + i wins
// (smallest duration, then smallest t0). LR >= 0, so its float bits order like uint.
__device__ __forceinline__ unsigned long long make_key(float lr, uint32_t flat) {
    return ((unsigned long long)__float_as_uint(lr) << 32) | (unsigned long long)(0xFFFFFFFFu - flat);
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
// The same copy to a 32-bit shared-memory address.
__device__ __forceinline__ void bulk_load_s(uint32_t dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
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
// Non-blocking test of a barrier phase (acquire: reads after a true result see the data).
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
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

}  // namespace
