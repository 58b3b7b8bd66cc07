// Warp scans and surrogates shared by the backward kernels (sm_103a).
// A warp holds 512 consecutive steps of one row, lane L steps 16L .. 16L+15.
#pragma once

#include "common.cuh"

namespace alif {

constexpr int BWD_E = 16;  // steps per lane

// Inclusive decayed prefix scan of q into V: V[t] = sum_{j<=t} b^{t-j} q[j].
// Blm[l] = b^(16*2^l) on lanes >= 2^l, 0 below; bm = b on lanes > 0, 0 on lane 0;
// b8 = b^8.  The lane's 16 steps are two 8-step chains (the second started from
// b^8 times the first's total), which halves the rounding depth of the in-lane
// passes (the recomputed V and a feed the surrogate, whose slope amplifies it).
__device__ __forceinline__ void scan16(const float (&q)[BWD_E], float (&V)[BWD_E], float b, float b8,
                                       const float (&Blm)[5], float bm) {
    float lo = q[0], hi = q[8];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        lo = fmaf(b, lo, q[k]);
        hi = fmaf(b, hi, q[8 + k]);
    }
    float tot = fmaf(b8, lo, hi);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = fmaf(Blm[l], __shfl_up_sync(FULL, tot, 1 << l), tot);
    const float P = __shfl_up_sync(FULL, tot, 1);
    const float P8 = fmaf(bm != 0.0f ? b8 : 0.0f, P, lo);  // V at the lane's step 7 (no carry into lane 0)
    V[0] = fmaf(bm, P, q[0]);
    V[8] = fmaf(b, P8, q[8]);
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        V[k] = fmaf(b, V[k - 1], q[k]);
        V[8 + k] = fmaf(b, V[8 + k - 1], q[8 + k]);
    }
}

// Inclusive reverse decayed scan in place: v[t] <- sum_{j>=t} b^{j-t} v[j].
// Brm[l] = b^(16*2^l) on lanes < 32 - 2^l, 0 above; bmr = b on lanes < 31, 0 on lane 31;
// b8 = b^8.  As in scan16 the lane's 16 steps are two 8-step chains: the upper half's value
// at its first step is rebuilt from the carry with the exact power b^8, so no contribution
// passes through more than eight multiplications by the rounded b.
__device__ __forceinline__ void rscan16(float (&v)[BWD_E], float b, float b8, const float (&Brm)[5], float bmr) {
    float lo = v[7], hi = v[BWD_E - 1];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        lo = fmaf(b, lo, v[k]);
        hi = fmaf(b, hi, v[8 + k]);
    }
    float tot = fmaf(b8, hi, lo);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = fmaf(Brm[l], __shfl_down_sync(FULL, tot, 1 << l), tot);
    const float P = __shfl_down_sync(FULL, tot, 1);
    const float P8 = fmaf(bmr != 0.0f ? b8 : 0.0f, P, hi);  // the sum at the lane's step 8
    v[BWD_E - 1] = fmaf(bmr, P, v[BWD_E - 1]);
#pragma unroll
    for (int k = BWD_E - 2; k >= 9; --k) v[k] = fmaf(b, v[k + 1], v[k]);
    v[8] = P8;
#pragma unroll
    for (int k = 7; k >= 0; --k) v[k] = fmaf(b, v[k + 1], v[k]);
}

// g_S times the surrogate dS/du at u = V - theta (Supplementary, "Surrogate gradient"):
// SG 0 fast sigmoid 1/(k|u|+1)^2; SG 1 multi-Gaussian 1.15 N(u|0, 0.5^2) - 0.15 N(u|3, 3^2)
// - 0.15 N(u|-3, 3^2) (N the normal density, as printed); SG 2 boxcar 0.5 on |u| <= 0.5.
template <int SG>
__device__ __forceinline__ float surrogate_times(float g, float u, float slope) {
    if (SG == 1) {
        const float c0 = 1.15f * 0.7978845608f;  // 1.15 / (0.5 sqrt(2 pi))
        const float c1 = 0.15f * 0.1329807601f;  // 0.15 / (3 sqrt(2 pi))
        const float up = u - 3.0f, um = u + 3.0f;
        const float sg = c0 * __expf(-2.0f * u * u) - c1 * (__expf(up * up * (-1.0f / 18.0f)) +
                                                              __expf(um * um * (-1.0f / 18.0f)));
        return g * sg;
    } else if (SG == 2) {
        return fabsf(u) <= 0.5f ? 0.5f * g : 0.0f;
    } else {
        const float den = fmaf(slope, fabsf(u), 1.0f);
        return __fdividef(g, den * den);
    }
}

}  // namespace alif
