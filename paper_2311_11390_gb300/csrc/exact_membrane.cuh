// Exact (double-single) membrane of one neuron row, shared by the block forward kernels: the
// re-decision of a spike whose FP32 margin lies inside the fast path's error bound.
#pragma once

#include "common.cuh"

namespace alif {

// Exact (double-single) membrane at global step t, from the anchor
// "V entering step anc_t equals anc_v" with no spike or mask in [anc_t, t]:
//   V[t] = beta^{t-anc_t+1} anc_v + sum_{j=anc_t}^{t} beta^{t-j} c I[j].
// Warp-cooperative: each lane takes a contiguous piece (Horner), pieces are
// scaled to t and summed with a butterfly (same result in every lane).
// COH: I is written by this kernel (fused projection), so it is read through L2 (coherent).
template <bool COH>
__device__ __noinline__ df exact_membrane(const float *__restrict__ Irow, long long anc_t,
                                          float anc_hi, float anc_lo, long long t, float bh,
                                          float bl, float ch, float cl, int lane) {
    const df beta{bh, bl}, c{ch, cl};
    const long long n = t - anc_t + 1;
    const long long len = (n + 31) >> 5;
    const long long lo = anc_t + (long long)lane * len;
    long long hi = lo + len;
    if (hi > t + 1) hi = t + 1;
    df h{0.0f, 0.0f};
    long long j = lo;
    for (; j + 8 <= hi; j += 8) {  // 8 loads in flight, then the 8 Horner steps in order
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = COH ? __ldcg(Irow + j + k) : __ldg(Irow + j + k);
#pragma unroll
        for (int k = 0; k < 8; ++k) h = df_add(df_mul(h, beta), df_mul_f(c, x[k]));
    }
    for (; j < hi; ++j) h = df_add(df_mul(h, beta), df_mul_f(c, COH ? __ldcg(Irow + j) : __ldg(Irow + j)));
    if (hi > lo) h = df_mul(h, df_pow(beta, t - (hi - 1)));
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const df o{__shfl_xor_sync(FULL, h.hi, off), __shfl_xor_sync(FULL, h.lo, off)};
        h = df_add(h, o);
    }
    return df_add(h, df_mul(df_pow(beta, n), df{anc_hi, anc_lo}));
}

}  // namespace alif
