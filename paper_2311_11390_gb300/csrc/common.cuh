// Shared device helpers for the ALIF kernels (sm_103a).
//
//  * double-single ("df") arithmetic: a value carried as an unevaluated sum of
//    two floats, built on the error-free transformations TwoSum (Knuth, TAOCP
//    vol. 2, 4.2.2) and TwoProduct via fused multiply-add (Dekker 1971 idea,
//    FMA form).  About 48 significant bits; used only where a spike decision
//    must match the FP64 standard model.
//  * PTX wrappers for mbarriers and the bulk (TMA, non-tensor) global->shared
//    copy, plus a globaltimer-bounded wait that never spins forever.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "alif.h"

namespace alif {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------ df arithmetic
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

// s + e == a + b exactly (any magnitudes).
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// s + e == a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

// p + e == a * b exactly (barring underflow).
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

// b^n by binary exponentiation (n >= 0).
__device__ __forceinline__ df df_pow(df b, long long n) {
    df r = df{1.0f, 0.0f};
    while (n > 0) {
        if (n & 1) r = df_mul(r, b);
        n >>= 1;
        if (n) b = df_mul(b, b);
    }
    return r;
}

// sign of a - b as a double-single difference: >0, 0, <0
__device__ __forceinline__ int df_cmp(df a, df b) {
    df d = df_add(a, df_neg(b));
    if (d.hi > 0.0f || (d.hi == 0.0f && d.lo > 0.0f)) return 1;
    if (d.hi < 0.0f || (d.hi == 0.0f && d.lo < 0.0f)) return -1;
    return 0;
}

// -------------------------------------------------------------- PTX helpers
// add + B * (src of lane - d) on lanes >= d, add on the others: the shuffle's own in-range
// predicate guards the FMA, so no per-lane table of factors (0 below d) is needed.
__device__ __forceinline__ float up_fma(float src, float B, unsigned d, float add) {
    float r;
    asm("{\n\t.reg .pred p;\n\t.reg .f32 u;\n\t"
        "shfl.sync.up.b32 u|p, %1, %2, 0, 0xffffffff;\n\t"
        "mov.f32 %0, %4;\n\t"
        "@p fma.rn.f32 %0, %3, u, %4;\n\t}"
        : "=f"(r)
        : "f"(src), "r"(d), "f"(B), "f"(add));
    return r;
}

// add + B * (src of lane + d) on lanes < 32 - d, add on the others.
__device__ __forceinline__ float down_fma(float src, float B, unsigned d, float add) {
    float r;
    asm("{\n\t.reg .pred p;\n\t.reg .f32 u;\n\t"
        "shfl.sync.down.b32 u|p, %1, %2, 31, 0xffffffff;\n\t"
        "mov.f32 %0, %4;\n\t"
        "@p fma.rn.f32 %0, %3, u, %4;\n\t}"
        : "=f"(r)
        : "f"(src), "r"(d), "f"(B), "f"(add));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, giving up after `limit_ns`.
// Returns false on timeout (the caller records ALIF_ETIMEOUT and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// 1-D bulk copy global -> shared, completion signalled on `bar` (tx bytes).
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Same with an L2 evict-first hint (data streamed once).
__device__ __forceinline__ void bulk_g2s_stream(void *dst, const void *src, uint32_t bytes,
                                                uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
        "%2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 32 x 32 bit-matrix transpose across the warp (recursive block swap): in, lane r
// holds row r (bit c = A[r][c]); out, lane r holds column r (bit c = A[c][r]).
__device__ __forceinline__ uint32_t bits_transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const int j = 16 >> l;
        const uint32_t m = masks[l];
        const uint32_t y = __shfl_xor_sync(FULL, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// The device status word lives in one translation unit (host.cu); kernels
// receive its address as an argument.
__device__ __forceinline__ void report_timeout(int *status) {
    if (status) atomicExch(status, ALIF_ETIMEOUT);
}

}  // namespace alif
