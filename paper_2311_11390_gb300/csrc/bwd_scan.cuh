// Warp scans and surrogates shared by the backward kernels (sm_103a).
#pragma once

#include "common.cuh"

namespace alif {

constexpr int BWD_E = 16;  // steps per lane of the attached backward (512-step windows)
constexpr int BWD8 = 8;    // steps per lane of the detached backward (256-step windows)

// Decayed scans of the detached backward, whose warp holds 256 consecutive steps of one
// row, lane L steps 8L .. 8L+7.  Spans of whole lanes, and of half lanes, decay by exact
// powers; inside a half lane by the rounded b.

// Inclusive decayed prefix scan of q into V: V[t] = sum_{j<=t} b^{t-j} q[j].
// Bk[l] = b^(8*2^l), b4 = b^4 (exact powers, rounded once).  The lane's 8 steps are two
// 4-step chains, the second restarted from b^4 times the carry into the lane plus the
// first's total, so no contribution passes through more than four multiplications by the
// rounded b (the recomputed V and a feed the surrogate, whose slope amplifies their rounding).
__device__ __forceinline__ void scan8(const float (&q)[BWD8], float (&V)[BWD8], float b, float b4,
                                      const float (&Bk)[5]) {
    float lo = q[0], hi = q[4];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        lo = fmaf(b, lo, q[k]);
        hi = fmaf(b, hi, q[4 + k]);
    }
    float tot = fmaf(b4, lo, hi);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = up_fma(tot, Bk[l], 1u << l, tot);
    const float P = up_fma(tot, 1.0f, 1u, 0.0f);  // V at the step before the lane's first (0 on lane 0)
    const float s3 = fmaf(b4, P, lo);  // V at the lane's step 3, from the exact power
    V[0] = fmaf(b, P, q[0]);
    V[4] = fmaf(b, s3, q[4]);
#pragma unroll
    for (int k = 1; k < 3; ++k) V[k] = fmaf(b, V[k - 1], q[k]);
    V[3] = s3;
#pragma unroll
    for (int k = 5; k < 8; ++k) V[k] = fmaf(b, V[k - 1], q[k]);
}

// Inclusive reverse decayed scan in place: v[t] <- sum_{j>=t} b^{j-t} v[j].  Bk, b4 and the
// two 4-step chains as in scan8.
__device__ __forceinline__ void rscan8(float (&v)[BWD8], float b, float b4, const float (&Bk)[5]) {
    float lo = v[3], hi = v[7];
#pragma unroll
    for (int k = 2; k >= 0; --k) {
        lo = fmaf(b, lo, v[k]);
        hi = fmaf(b, hi, v[4 + k]);
    }
    float tot = fmaf(b4, hi, lo);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = down_fma(tot, Bk[l], 1u << l, tot);
    const float P = down_fma(tot, 1.0f, 1u, 0.0f);  // the sum at the step after the lane's last (0 on lane 31)
    const float s4 = fmaf(b4, P, hi);  // the sum at the lane's step 4, from the exact power
    v[7] = fmaf(b, P, v[7]);
    v[3] = fmaf(b, s4, v[3]);
#pragma unroll
    for (int k = 6; k > 4; --k) v[k] = fmaf(b, v[k + 1], v[k]);
    v[4] = s4;
#pragma unroll
    for (int k = 2; k >= 0; --k) v[k] = fmaf(b, v[k + 1], v[k]);
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
