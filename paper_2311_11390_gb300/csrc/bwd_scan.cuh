// Warp scans and surrogates shared by the backward kernels (sm_103a).
#pragma once

#include "common.cuh"

namespace alif {

constexpr int BWD_E = 16;  // steps per lane of the attached backward (512-step windows)

// Decayed scans of the detached backward, whose warp holds 32 E consecutive steps of one row,
// lane L steps E L .. E L + E - 1 (E = 8 or 16).  Each lane's steps are two chains of H = E / 2;
// spans of whole lanes, and of half lanes, decay by exact powers, inside a half lane by the
// rounded b, so no contribution passes through more than H multiplications by the rounded b
// (the recomputed V and a feed the surrogate, whose slope amplifies their rounding).

// Inclusive decayed prefix scan of q into V: V[t] = sum_{j<=t} b^{t-j} q[j].
// Bk[l] = b^(E 2^l), bh = b^H (exact powers, rounded once).
template <int E>
__device__ __forceinline__ void scan_lane(const float (&q)[E], float (&V)[E], float b, float bh,
                                          const float (&Bk)[5]) {
    constexpr int H = E / 2;
    float lo = q[0], hi = q[H];
#pragma unroll
    for (int k = 1; k < H; ++k) {
        lo = fmaf(b, lo, q[k]);
        hi = fmaf(b, hi, q[H + k]);
    }
    float tot = fmaf(bh, lo, hi);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = up_fma(tot, Bk[l], 1u << l, tot);
    const float P = up_fma(tot, 1.0f, 1u, 0.0f);  // V at the step before the lane's first (0 on lane 0)
    const float sh = fmaf(bh, P, lo);             // V at the lane's step H - 1, from the exact power
    V[0] = fmaf(b, P, q[0]);
    V[H] = fmaf(b, sh, q[H]);
#pragma unroll
    for (int k = 1; k < H - 1; ++k) V[k] = fmaf(b, V[k - 1], q[k]);
    V[H - 1] = sh;
#pragma unroll
    for (int k = H + 1; k < E; ++k) V[k] = fmaf(b, V[k - 1], q[k]);
}

// Inclusive reverse decayed scan in place: v[t] <- sum_{j>=t} b^{j-t} v[j].  Bk, bh and the
// two half-lane chains as in scan_lane.
template <int E>
__device__ __forceinline__ void rscan_lane(float (&v)[E], float b, float bh, const float (&Bk)[5]) {
    constexpr int H = E / 2;
    float lo = v[H - 1], hi = v[E - 1];
#pragma unroll
    for (int k = H - 2; k >= 0; --k) {
        lo = fmaf(b, lo, v[k]);
        hi = fmaf(b, hi, v[H + k]);
    }
    float tot = fmaf(bh, hi, lo);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = down_fma(tot, Bk[l], 1u << l, tot);
    const float P = down_fma(tot, 1.0f, 1u, 0.0f);  // the sum at the step after the lane's last (0 on lane 31)
    const float sh = fmaf(bh, P, hi);               // the sum at the lane's step H, from the exact power
    v[E - 1] = fmaf(b, P, v[E - 1]);
    v[H - 1] = fmaf(b, sh, v[H - 1]);
#pragma unroll
    for (int k = E - 2; k > H; --k) v[k] = fmaf(b, v[k + 1], v[k]);
    v[H] = sh;
#pragma unroll
    for (int k = H - 2; k >= 0; --k) v[k] = fmaf(b, v[k + 1], v[k]);
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
