// ARP-blocked ALIF forward (Section 3, Props 1-5) for sm_103a.
//
// One warp simulates one neuron row at a time and walks time in windows of
// WIN = 256 steps (one checkpoint stride), lane L holding steps 8L..8L+7 of the
// window.  A window is resolved in "rounds":
//   1. the no-reset membrane of Prop 1 over the admitted part of the window,
//      V~[t] = beta^{t+1} v_in + sum_{j<=t} beta^{t-j} (1-beta) R I[j],
//      is a decayed prefix scan: each lane folds its 8 inputs into one
//      total, a 5-level shuffle scan carries the totals across lanes, and a
//      second in-lane pass rebuilds the 8 prefix values from the carry;
//   2. the adaptive threshold is theta0 + d p^t a_w (Prop 5, no spike yet);
//   3. the first crossing V~ > theta (Props 2 and Eq 9: only the first faulty
//      spike is real) is found with a warp ballot and __ffs;
//   4. after a spike at tau the membrane is reset (Prop 4) and input is masked
//      until tau + T_eff (Prop 3), so the next round rescans from there with a
//      zero start; the adaptation restarts from a[tau+1] = p a[tau] + 1 (Prop 5).
// A window without spikes costs one round however many T_R-blocks it spans.
// The state entering each window is its checkpoint.  Eight steps per lane keep
// the window's register arrays small enough for four CTAs of four warps per SM:
// the kernel is bound by the latency of its scan and candidate chains, and the
// extra warps hide it.
//
// Input staging: when T is a multiple of 16 the current is viewed as rows of
// 16 floats and each window (16 such rows) is one 2-D TMA box with 64-byte
// swizzle, so that the lanes' 16-byte reads hit distinct bank groups;
// otherwise lanes read global memory directly.
//
// Exactness of the spike decisions: the FP32 margin M = V~ - theta comes with
// an error bound G, and |M| <= G is re-decided in double-single arithmetic from
// an exact anchor (the last reset, where V is exactly 0, or the last re-decided
// step), re-reading the inputs since the anchor from global memory.  Decisions
// then agree with the FP64 standard model except for margins ~1e-13.  The bound,
// with u = 2^-24 and W = 32 E steps per window: along any path through the scan a
// term of V~ meets at most E + 16 roundings (the lane's chain 2k + 2, the lane
// total 2, five shuffle levels 2 each, the rebuild 2 or 4, counting the rounded
// powers of beta and c), so V~ errs by at most (E + 16) u (beta^(t+1) |v_in| +
// R (1 - beta^(t+1)) max|I|) <= (E + 16) u max(|v_in|, R max_win|I|); the entering
// membrane is carried in FP32, so earlier windows' errors, decaying by beta^W, add
// at most (E + 16) u (beta^W / (1 - beta^W) max_row|v_in| + R max_row|I|); d a's
// three roundings, the margin's FMA and theta0 - G add u (4 |d a| + |V~| + theta0).
// G is that sum times 1 + 2^-6 (the second-order terms and G's own evaluation); a
// rescan after a spike starts from an exact 0 and carries no earlier error.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "common.cuh"
#include "exact_membrane.cuh"
#include "tmap.h"

namespace alif {
namespace fwd {

constexpr int WARPS = 4;  // warps per CTA
#ifndef ALIF_FWD_MIN_BLOCKS
#define ALIF_FWD_MIN_BLOCKS 4  // CTAs per SM the register budget of the 256-step kernel is sized for
#endif
// per warp: the TMA ring, or (fused projection) the neuron's FP32 weight row of up to 1024 inputs
constexpr int RING_WARP_BYTES = 4096;
static_assert(RING_WARP_BYTES >= 1024 * 4, "the ring area holds a weight row of the fused projection");
constexpr int RING_BYTES = WARPS * RING_WARP_BYTES;
constexpr int HALF = ALIF_CKPT_STEPS;  // checkpoint stride
// Window geometry for E steps per lane: E = 8, 256-step windows (one checkpoint stride), four CTAs
// per SM; E = 16, 512-step windows (two strides: the state entering the middle step is recorded
// as the round covering it is resolved), three CTAs per SM.
template <int E>
struct Geo {
    static_assert(E == 8 || E == 16, "8 or 16 steps per lane");
    static constexpr int WIN = 32 * E;
    static constexpr int H = E / 2;
    static constexpr int CK = WIN / HALF;                         // checkpoints per window
    static constexpr int STAGE_BYTES = WIN * 4;
    static constexpr int NSTAGE = RING_WARP_BYTES / STAGE_BYTES;  // TMA ring depth: 4 or 2
    static constexpr int PDN = WIN + 4;                           // p^j, j = 0..WIN, padded to 16-byte rows
    static constexpr int PD_BYTES = WARPS * 2 * PDN * 4;          // p^j double-single tables
    // per-warp row constants: beta^1..beta^H at 0, beta^(E 2^l) at 8..12, p^(E-1) at 13
    static constexpr int RT_FLOATS = 16;
    static constexpr int SMEM_BYTES = RING_BYTES + PD_BYTES + WARPS * RT_FLOATS * 4 + WARPS * NSTAGE * 8 + 1024;
    static constexpr int MIN_BLOCKS = E == 8 ? ALIF_FWD_MIN_BLOCKS : 3;
    static_assert((RING_BYTES + PD_BYTES) % 16 == 0 && (RT_FLOATS * 4) % 16 == 0,
                  "row tables 16-byte aligned (float2 reads), barriers 8-byte aligned");
};

struct Args {
    long long rows, N, T, nwords, nckpt, nwin;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    uint32_t *spikes;
    float *vtr, *atr;
    AlifState *ckpt, *fin;
    unsigned long long *counters;  // [0] re-decided margins, [1] of which spikes, [2] rows
    int *status;
    // fused projection (LOAD 2): I is computed from the input events and written to `I`
    const float *W, *bias;         // [N, Nin] FP32 weights, [N] bias (nullable)
    const int *ev_off;             // [B * nw_in, EV_ROW] per-step event offsets of each 32-step word
    const uint16_t *ev_ent;        // [B * nw_in, ev_cap] active inputs, by step then input
    long long Nin, nw_in;
    int ev_cap;
};
constexpr int EV_ROW = 36;  // ints per word: offsets of steps 0..32, padded to 16-byte rows

// Bits k of a lane (steps t0 + k) with lo <= t0 + k < hi.
template <int E>
__device__ __forceinline__ unsigned lane_bits(int lo, int hi, int t0) {
    const int h = min(max(hi - t0, 0), E), l = min(max(lo - t0, 0), E);
    return ((1u << h) - 1u) & ~((1u << l) - 1u);
}

// Inclusive decayed prefix scan of q over the warp's 32 E steps into V:
// V[t] = sum_{j<=t} b^{t-j} q[j] (lane 0 carries nothing in; a window's entering membrane
// is folded into its q[0] by the caller).  Pass 1: the lane's two H-step chains from zero
// (L, H = E / 2); a 5-level shuffle scan of the lane totals (Bl[l] = b^(E 2^l), applied on the
// lanes the shuffle reaches) gives P, the membrane entering the lane.  Pass 2 adds the carries
// with the exact powers Bk2 = (b, b^2), (b^3, b^4), ... up to b^H as packed f32x2 FMAs:
// V[k] = L[k] + b^(k+1) P for k < H and V[k] = L[k] + b^(k-H+1) V[H-1] above.  No contribution
// passes through more than H multiplications by the rounded b.
template <int E>
__device__ __forceinline__ void scan_win(const float (&q)[E], float (&V)[E], float b, float bh, const float *Bl,
                                         const float2 *Bk2) {
    constexpr int H = E / 2;
    float L[E];
    L[0] = q[0];
    L[H] = q[H];
#pragma unroll
    for (int k = 1; k < H; ++k) {
        L[k] = fmaf(b, L[k - 1], q[k]);
        L[H + k] = fmaf(b, L[H + k - 1], q[H + k]);
    }
    float tot = fmaf(bh, L[H - 1], L[E - 1]);
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = up_fma(tot, Bl[l], 1u << l, tot);
    const float P = up_fma(tot, 1.0f, 1u, 0.0f);  // V at the step before this lane's first (0 on lane 0)
    const float2 PP = make_float2(P, P);
#pragma unroll
    for (int j = 0; j < H / 2; ++j) {
        const float2 v = __ffma2_rn(Bk2[j], PP, make_float2(L[2 * j], L[2 * j + 1]));
        V[2 * j] = v.x;
        V[2 * j + 1] = v.y;
    }
    const float2 QQ = make_float2(V[H - 1], V[H - 1]);
#pragma unroll
    for (int j = 0; j < H / 2; ++j) {
        const float2 w = __ffma2_rn(Bk2[j], QQ, make_float2(L[H + 2 * j], L[H + 2 * j + 1]));
        V[H + 2 * j] = w.x;
        V[H + 2 * j + 1] = w.y;
    }
}

// v[k] by a select tree on the bits of k (0 <= k < E).
template <int E>
__device__ __forceinline__ float pick(const float (&v)[E], int k) {
    float a[E / 2];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) a[i] = (k & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int w = E / 4, bit = 2; w >= 1; w /= 2, bit *= 2) {
#pragma unroll
        for (int i = 0; i < w; ++i) a[i] = (k & bit) ? a[2 * i + 1] : a[2 * i];
    }
    return a[0];
}

// Bits k of the steps whose Z[k] >= thr (a balanced tree of ORs).
template <int E>
__device__ __forceinline__ unsigned cand(const float (&Z)[E], float thr) {
    unsigned m[E / 2];
#pragma unroll
    for (int i = 0; i < E / 2; ++i)
        m[i] = (Z[2 * i] >= thr ? 1u << (2 * i) : 0u) | (Z[2 * i + 1] >= thr ? 2u << (2 * i) : 0u);
#pragma unroll
    for (int w = E / 4; w >= 1; w /= 2) {
#pragma unroll
        for (int i = 0; i < w; ++i) m[i] = m[2 * i] | m[2 * i + 1];
    }
    return m[0];
}

// Z[k] = V[k] - dA P[k] as packed f32x2 FMAs.
template <int E>
__device__ __forceinline__ void margins(const float (&V)[E], float dA, const float (&P)[E], float (&Z)[E]) {
    const float2 nd = make_float2(-dA, -dA);
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
        const float2 z = __ffma2_rn(nd, make_float2(P[2 * j], P[2 * j + 1]), make_float2(V[2 * j], V[2 * j + 1]));
        Z[2 * j] = z.x;
        Z[2 * j + 1] = z.y;
    }
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Maximum of E values with three-input max instructions.
template <int E>
__device__ __forceinline__ float vmax(const float (&v)[E]) {
    if constexpr (E == 8) {
        return fmax3(fmax3(v[0], v[1], v[2]), fmax3(v[3], v[4], v[5]), fmaxf(v[6], v[7]));
    } else {
        const float a = fmax3(v[0], v[1], v[2]), b = fmax3(v[3], v[4], v[5]), c = fmax3(v[6], v[7], v[8]);
        const float d = fmax3(v[9], v[10], v[11]), e = fmax3(v[12], v[13], v[14]);
        return fmaxf(fmax3(a, b, c), fmax3(d, e, v[15]));
    }
}

// Maximum of |v| over E values.
template <int E>
__device__ __forceinline__ float vabsmax(const float (&v)[E]) {
    float m[E / 2];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) m[i] = fmaxf(fabsf(v[2 * i]), fabsf(v[2 * i + 1]));
    if constexpr (E == 8) {
        return fmax3(m[0], m[1], fmaxf(m[2], m[3]));
    } else {
        return fmax3(fmax3(m[0], m[1], m[2]), fmax3(m[3], m[4], m[5]), fmaxf(m[6], m[7]));
    }
}

// LOAD: 1 = 2-D TMA ring, 0 = direct global loads, 2 = fused projection (I computed from the input
// events and the FP32 weight row staged in the warp's ring area, then written out)
template <int LOAD, bool VTR, bool ATR, int E>
__global__ void __launch_bounds__(WARPS * 32, Geo<E>::MIN_BLOCKS)
    fwd_kernel(const __grid_constant__ CUtensorMap tm, const Args A) {
    constexpr int WIN = Geo<E>::WIN, H = Geo<E>::H, CK = Geo<E>::CK, NSTAGE = Geo<E>::NSTAGE;
    constexpr int STAGE_BYTES = Geo<E>::STAGE_BYTES, PDN = Geo<E>::PDN, PD_BYTES = Geo<E>::PD_BYTES;
    constexpr int RT_FLOATS = Geo<E>::RT_FLOATS;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // swizzled stages: 1024-aligned
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(sm + warp * RING_WARP_BYTES);
    float *pdh = reinterpret_cast<float *>(sm + RING_BYTES) + warp * 2 * PDN;  // p^j hi, j=0..WIN
    float *pdl = pdh + PDN;                                                   // p^j lo
    // the row's span decays, read by every lane (kept out of the registers): beta^1 .. beta^H
    // (8-byte aligned pairs), beta^(E 2^l) for a span of 2^l lanes (l = 0..4), p^(E-1)
    float *rt = reinterpret_cast<float *>(sm + RING_BYTES + PD_BYTES) + warp * RT_FLOATS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + RING_BYTES + PD_BYTES + WARPS * RT_FLOATS * 4) + warp * NSTAGE;
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long nw = (long long)gridDim.x * WARPS;
    if (gw >= A.rows) return;  // warps are independent: no block-level barrier below

    // ---- TMA producer (lane 0 issues; every lane tracks the cursor)
    long long p_row = gw;
    int p_wi = 0;
    const int nwin = (int)A.nwin;
    const int lastcnt = (int)(A.T - (long long)(nwin - 1) * WIN);
    unsigned issued = 0, consumed = 0;
    if (LOAD == 1) {
        if (lane == 0) {
            for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    auto issue = [&]() {
        while (p_row < A.rows && issued - consumed < (unsigned)NSTAGE) {
            if (lane == 0) {
                const int st = issued % NSTAGE;
                mbar_arrive_expect_tx(&bars[st], STAGE_BYTES);
                tma_load_2d_u(smem_u32(ring + st * WIN), &tm, 0,
                              (int)((p_row * A.T + (long long)p_wi * WIN) >> 4), smem_u32(&bars[st]));
            }
            ++issued;
            if (++p_wi == nwin) {
                p_wi = 0;
                p_row += nw;
            }
        }
    };
    if (LOAD == 1) issue();

    bool dead = false;
    unsigned n_exact = 0, n_exact_spk = 0, n_rows = 0;
    const int t0 = E * lane;
    // this lane's E floats of a stage: 16-byte chunks ch0 .. ch0 + E/4 - 1 of box row t0 / 16, under
    // the 64-byte swizzle of that row (a quarter warp's 16-byte reads fall in distinct bank groups)
    const int swz = ((t0 >> 4) >> 1) & 3, ch0 = (t0 & 15) >> 2, brow = 16 * (t0 >> 4);

    for (long long r = gw; r < A.rows && !dead; r += nw) {
        const AlifNeuron nr = A.nrn[r % A.N];
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        const float *Irow = A.I + r * A.T;
        float bias_i = 0.0f;
        if (LOAD == 2) {
            // the neuron's FP32 weight row into the warp's ring area (the fused path has no TMA ring)
            const float *Wrow = A.W + (r % A.N) * A.Nin;
            for (long long j = lane; j < A.Nin; j += 32) ring[j] = __ldg(Wrow + j);
            if (A.bias) bias_i = __ldg(A.bias + r % A.N);
            __syncwarp();
        }
        const float bf = nr.beta_hi, pf = nr.p_hi, c = nr.c_hi;

        // Warp tables: p^j (j = 0..WIN) as double-single pairs; span decays.
        float Pw0;  // p^{t0}
        {
            df q = df_pow(p, t0);
            Pw0 = q.hi;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                pdh[t0 + k] = q.hi;
                pdl[t0 + k] = q.lo;
                q = df_mul(q, p);
            }
            if (lane == 31) {
                pdh[WIN] = q.hi;
                pdl[WIN] = q.lo;
            }
            if (lane < H) rt[lane] = df_pow(beta, lane + 1).hi;
            else if (lane >= 8 && lane < 13) rt[lane] = df_pow(beta, (long long)E << (lane - 8)).hi;
            else if (lane == 13) rt[13] = df_pow(p, E - 1).hi;
        }
        __syncwarp();
        const float2 *Bk2 = reinterpret_cast<const float2 *>(rt);  // (beta, beta^2), (beta^3, beta^4), ...
        const float *Bl = rt + 8;                                   // beta^(E 2^l)
        const float bhf = rt[H - 1];                                // beta^H
        auto pdf = [&](int j) { return df{pdh[j], pdl[j]}; };
        // error bound factors (header), u' = u (1 + 2^-6): G = gM max(|v_in|, R max_win|I|) + gD |d a|
        // + g0 (+ gC max_row|v_in| + gR max_row|I| for a window's first round); the carried factor
        // beta^W / (1 - beta^W) from double-single beta^W, capped at 2^20 (G then covers any margin)
        constexpr float us = 5.9604645e-8f * 1.015625f;
        float gC;
        {
            const df bw = df_pow(beta, WIN);
            const float om = (1.0f - bw.hi) - bw.lo;
            gC = (E + 16.0f) * us * fminf(bw.hi / fmaxf(om, 0x1p-20f), 0x1p20f);
        }
        const float gM = (E + 17.0f) * us, gD = 4.0f * us, gR = (E + 16.0f) * us * nr.R, g0 = us * nr.theta0;

        // ---- state entering the row
        float Vin;
        df aw;
        int rel;  // input masked (refractory) for window steps < rel
        long long anc_t;
        df anc_v;
        {
            AlifState s0{0.0f, 0.0f, 0};
            if (A.init) s0 = A.init[r];
            const int rem = s0.rem > 0 ? s0.rem : 0;
            Vin = rem > 0 ? 0.0f : s0.v;
            aw = df{s0.a, 0.0f};
            rel = rem;
            anc_t = rem;
            anc_v = df{Vin, 0.0f};
        }
        float mxr = 0.0f, vmr = 0.0f;  // running maxima of |I| and of the entering membrane's |v_in|

        for (int wi = 0; wi < nwin; ++wi) {
            const long long w = (long long)wi * WIN;
            const bool last = wi == nwin - 1;
            const int cnt = last ? lastcnt : WIN;
            float cx[E];
            if (LOAD == 1) {
                const int st = consumed % NSTAGE;
                if (!mbar_wait_bounded(&bars[st], (consumed / NSTAGE) & 1u)) {
                    report_timeout(A.status);
                    dead = true;
                    break;
                }
                const float *row16 = ring + st * WIN + brow;  // the box row holding this lane's steps
#pragma unroll
                for (int q = 0; q < E / 4; ++q) {
                    const float4 u = *reinterpret_cast<const float4 *>(row16 + 4 * ((ch0 + q) ^ swz));
                    cx[4 * q] = u.x; cx[4 * q + 1] = u.y; cx[4 * q + 2] = u.z; cx[4 * q + 3] = u.w;
                }
                __syncwarp();
                fence_proxy_async_smem();
                ++consumed;
                issue();
            } else if (LOAD == 2) {
                // I[t] = bias + sum of the weights of the inputs active at t, in ascending input
                // order (Eq 3's feedforward term); this lane's E steps are part of a 32-step word,
                // whose per-step event offsets come in one 16-byte-aligned row.
                // Lanes whose steps all lie past T (last window) read nothing: their word does not exist
                const bool has = t0 < cnt;
                const long long wg = has ? (w + t0) >> 5 : 0;
                const long long bw = (r / A.N) * A.nw_in + wg;
                int o[E + 1];
#pragma unroll
                for (int k = 0; k <= E; ++k) o[k] = 0;
                if (has) {
                    const int *orow = A.ev_off + bw * EV_ROW + (t0 & 31);
#pragma unroll
                    for (int q = 0; q < E / 4; ++q) {
                        const int4 v = __ldg(reinterpret_cast<const int4 *>(orow) + q);
                        o[4 * q] = v.x; o[4 * q + 1] = v.y; o[4 * q + 2] = v.z; o[4 * q + 3] = v.w;
                    }
                    o[E] = __ldg(orow + E);
                }
                const uint16_t *ep = A.ev_ent + bw * A.ev_cap;
                int e = min(o[0], A.ev_cap);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    float acc = bias_i;
                    const int ee = min(o[k + 1], A.ev_cap);
                    for (; e < ee; ++e) acc += ring[__ldg(ep + e)];
                    cx[k] = (t0 + k < cnt) ? acc : 0.0f;
                }
                // written out for the backward (and re-read by the exact re-decisions below)
                float *Io = const_cast<float *>(Irow) + w + t0;
                if (t0 + E <= cnt && (A.T & 3) == 0) {
#pragma unroll
                    for (int q = 0; q < E / 4; ++q)
                        reinterpret_cast<float4 *>(Io)[q] = make_float4(cx[4 * q], cx[4 * q + 1], cx[4 * q + 2], cx[4 * q + 3]);
                } else {
#pragma unroll
                    for (int k = 0; k < E; ++k)
                        if (t0 + k < cnt) Io[k] = cx[k];
                }
                __syncwarp();  // the window's currents are visible to the warp's exact re-reads
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) cx[k] = (t0 + k < cnt) ? __ldg(Irow + w + t0 + k) : 0.0f;
            }
            if (last) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (t0 + k >= cnt) cx[k] = 0.0f;
            }
            const int s1 = rel <= 0 ? 0 : (rel >= cnt ? cnt : rel);

            if (A.ckpt && lane == 0) {  // the state entering the window (checkpoint CK wi)
                AlifState cs;
                cs.v = Vin;
                cs.a = aw.hi;
                cs.rem = rel > 0 ? rel : 0;
                A.ckpt[r * A.nckpt + (long long)CK * wi] = cs;
            }

            // Scale of the error bound.  V is a convex combination of v_in and
            // R I[j], so |V| <= max(|v_in|, R max|I|); errors carried from earlier
            // windows are bounded through the row's running maxima.  |x| is
            // non-negative, so its bit pattern orders like the value (integer max).
            float mx = vabsmax<E>(cx);
            mx = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(mx)));
            mxr = fmaxf(mx, mxr);
            vmr = fmaxf(vmr, fabsf(Vin));
            const float Rmx = nr.R * mx;

            // c I (masked before s1); cx keeps it for the rescans after spikes
            if (s1 == 0) {
                const float2 cc = make_float2(c, c);
#pragma unroll
                for (int j = 0; j < E / 2; ++j) {
                    const float2 v = __fmul2_rn(cc, make_float2(cx[2 * j], cx[2 * j + 1]));
                    cx[2 * j] = v.x;
                    cx[2 * j + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) cx[k] = (t0 + k >= s1) ? c * cx[k] : 0.0f;
            }

            float V[E], Z[E], vt[E], a_el[E];
            // ---- first round: no spike since the window start (a = p^t a_w).  The
            // entering membrane joins the scan as beta v_in added to step 0.
            float G = fmaf(gM, fmaxf(fabsf(Vin), Rmx), fmaf(gD, fabsf(nr.d * aw.hi), fmaf(gC, vmr, fmaf(gR, mxr, g0))));
            float thr = nr.theta0 - G;  // Z[k] = V - d a; a candidate where Z >= thr
            float zlim;
            {
                float q0[E];
#pragma unroll
                for (int k = 0; k < E; ++k) q0[k] = cx[k];
                if (lane == 0) q0[0] = fmaf(bf, Vin, q0[0]);
                scan_win<E>(q0, V, bf, bhf, Bl, Bk2);
                // d a = s p^k over the lane's steps (s = d a_w p^{t0}), so V - d a <= max V -
                // min(s, s p^(E-1)): one vote on that bound decides whether any step needs its
                // margin (usually none).  The bound's own roundings against those of the margins
                // are at most 3u |max V - min| + 5u |s|: 8u (|.| + |s|) plus a quarter of G cover them.
                const float sa = nr.d * aw.hi * Pw0;
                const float zb0 = vmax<E>(V) - fminf(sa, sa * rt[13]);
                zlim = zb0 + fmaf(8.0f * 5.9604645e-8f, fabsf(zb0) + fabsf(sa), 0.25f * G);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    if (VTR) vt[k] = V[k];
                    if (ATR) a_el[k] = pdh[t0 + k] * aw.hi;
                }
            }
            unsigned zb = 0;
            bool any = __any_sync(FULL, zlim >= thr);
            if (any) {
                // d a = d a_w p^t, with p^t from the table (16-byte reads of the lane's steps);
                // a candidate where V - d a >= theta0 - G
                float P[E];
#pragma unroll
                for (int q = 0; q < E / 4; ++q) {
                    const float4 u = *reinterpret_cast<const float4 *>(pdh + t0 + 4 * q);
                    P[4 * q] = u.x; P[4 * q + 1] = u.y; P[4 * q + 2] = u.z; P[4 * q + 3] = u.w;
                }
                margins<E>(V, nr.d * aw.hi, P, Z);
                zb = cand<E>(Z, thr) & lane_bits<E>(s1, cnt, t0);
                any = __any_sync(FULL, zb != 0u);
            }

            uint32_t sword = 0;
            int last_tau = -1, s2 = 0, aanc_rel = 0;
            df aanc = aw, A1{0.0f, 0.0f};
            // 512-step windows: the state entering the window's middle step (checkpoint CK wi + 1),
            // recorded from the round that covers it, before a later spike rescans the window
            int s_cur = rel;  // first step the current round's V is valid for (unclamped)
            bool mid_done = !(CK == 2 && A.ckpt && cnt > HALF);
            auto capture_mid = [&]() {
                const float vmid = __shfl_sync(FULL, V[E - 1], HALF / E - 1);
                if (lane == 0) {
                    AlifState cs;
                    cs.v = s_cur <= HALF - 1 ? vmid : 0.0f;
                    cs.a = df_mul(pdf(HALF - aanc_rel), aanc).hi;
                    cs.rem = s_cur > HALF ? s_cur - HALF : 0;
                    A.ckpt[r * A.nckpt + (long long)CK * wi + 1] = cs;
                }
                mid_done = true;
            };
            if (any) {
                // ---- resolve crossings in order: exact re-decision inside the
                // error band, spike, reset + ARP skip, rescan
                while (true) {
                    // each lane's first candidate and its margin, then the first lane holding one
                    const int myk = __ffs(zb) - 1;
                    const float myz = pick<E>(Z, myk & (E - 1));
                    const unsigned bal = __ballot_sync(FULL, zb != 0u);
                    if (bal == 0u) break;
                    const int Lf = __ffs(bal) - 1;
                    const int kf = __shfl_sync(FULL, myk, Lf);
                    const float zf = __shfl_sync(FULL, myz, Lf) - thr;  // V - theta + G
                    const int tf = E * Lf + kf;
                    if (CK == 2 && !mid_done && tf >= HALF) capture_mid();
                    if (!(zf > 2.0f * G)) {
                        // margin within the FP32 error bound: decide exactly
                        ++n_exact;
                        const long long tg = w + tf;
                        const df Vx = exact_membrane<LOAD == 2>(Irow, anc_t, anc_v.hi, anc_v.lo, tg, nr.beta_hi,
                                                                nr.beta_lo, nr.c_hi, nr.c_lo, lane);
                        const df ax = df_mul(pdf(tf - aanc_rel), aanc);
                        const df thx = df_add(df_mul_f(ax, nr.d), df{nr.theta0, 0.0f});
                        if (df_cmp(Vx, thx) <= 0) {
                            anc_t = tg + 1;  // exact V is now known entering tg + 1
                            anc_v = Vx;
                            if (lane == Lf) zb &= ~((2u << kf) - 1u);
                            continue;
                        }
                        ++n_exact_spk;
                    }
                    // ---- spike at tau (first crossing of this round)
                    const int tau = tf;
                    if (lane == (tau >> 5)) sword |= 1u << (tau & 31);
                    const df a_tau = df_mul(pdf(tau - aanc_rel), aanc);
                    A1 = df_add(df_mul(p, a_tau), df{1.0f, 0.0f});  // a[tau+1] (Eq 5)
                    aanc_rel = tau + 1;
                    aanc = A1;
                    last_tau = tau;
                    s2 = tau + nr.teff;  // input admitted again from here (Eq 4)
                    s_cur = s2;
                    rel = s2;
                    anc_t = w + s2;  // V is exactly 0 entering w + s2
                    anc_v = df{0.0f, 0.0f};
                    // a[t] = p^{t-tau-1} A1 for t > tau
                    const int t1 = tau + 1;
                    if (ATR || VTR) {
                        // the traces: per lane a chain of p from pb0 = p^{t0-tau-1} (lanes after tau's
                        // successor), restarted at 1 in the lane holding tau + 1
                        const int Lq = t1 / E, kq = t1 & (E - 1);
                        const float vB = __shfl_sync(FULL, Pw0, (lane - Lq - 1) & 31);
                        const float pb0 = lane > Lq ? vB * pdh[E - kq] : 0.0f;
                        const int kst = lane == Lq ? kq : -1;
                        float pk = pb0;
#pragma unroll
                        for (int k = 0; k < E; ++k) {
                            if (k == kst) pk = 1.0f;
                            if (t0 + k > tau) {
                                if (ATR) a_el[k] = pk * A1.hi;
                                if (VTR) vt[k] = 0.0f;
                            }
                            pk *= pf;
                        }
                    }
                    if (s2 >= cnt) break;
                    const float dA = nr.d * A1.hi;
                    const int Ls = s2 / E;  // first lane holding admitted steps
                    {
                        // rescan from s2 with a zero start (Props 1, 3, 4)
                        G = fmaf(gM, Rmx, fmaf(gD, fabsf(dA), g0));  // from an exact 0: no carried error
                        float q[E];
#pragma unroll
                        for (int k = 0; k < E; ++k) q[k] = (t0 + k >= s2) ? cx[k] : 0.0f;
                        scan_win<E>(q, V, bf, bhf, Bl, Bk2);
                    }
                    thr = nr.theta0 - G;
                    {
                        // d a[t] = dA p^{t - t1} from the table (steps before t1 are masked, and
                        // their V is 0 in this round: the clamped power keeps their Z below thr)
                        float P[E];
#pragma unroll
                        for (int k = 0; k < E; ++k) P[k] = pdh[max(t0 + k - t1, 0)];
                        margins<E>(V, dA, P, Z);
                    }
                    if (VTR) {
#pragma unroll
                        for (int k = 0; k < E; ++k)
                            if (t0 + k >= s2) vt[k] = V[k];
                    }
                    // usually no step of the rest of the window comes near theta: one vote on the
                    // lanes' maxima (lanes wholly before s2 abstain) instead of E compares
                    zb = 0;
                    if (__any_sync(FULL, lane >= Ls && vmax<E>(Z) >= thr))
                        zb = cand<E>(Z, thr) & lane_bits<E>(s2, cnt, t0);
                }
            }
            if (CK == 2 && !mid_done) capture_mid();

            // ---- outputs of the window
            if (lane < WIN / 32) {
                const long long widx = (long long)wi * (WIN / 32) + lane;
                if (widx < A.nwords) A.spikes[r * A.nwords + widx] = sword;
            }
            if (VTR || ATR) {
                float *vo = VTR ? A.vtr + r * A.T + w + t0 : nullptr;
                float *ao = ATR ? A.atr + r * A.T + w + t0 : nullptr;
                if (LOAD == 1 && t0 + E <= cnt) {
#pragma unroll
                    for (int q = 0; q < E / 4; ++q) {
                        if (VTR)
                            reinterpret_cast<float4 *>(vo)[q] =
                                make_float4(vt[4 * q], vt[4 * q + 1], vt[4 * q + 2], vt[4 * q + 3]);
                        if (ATR)
                            reinterpret_cast<float4 *>(ao)[q] =
                                make_float4(a_el[4 * q], a_el[4 * q + 1], a_el[4 * q + 2], a_el[4 * q + 3]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        if (t0 + k < cnt) {
                            if (VTR) vo[k] = vt[k];
                            if (ATR) ao[k] = a_el[k];
                        }
                    }
                }
            }

            // ---- carry to the next window (Props 4 and 5)
            float Vnext;
            {
                float mine = V[E - 1];
                if (last) {
                    const int kl = (cnt - 1) & (E - 1);
#pragma unroll
                    for (int k = 0; k < E - 1; ++k)
                        if (k == kl) mine = V[k];
                }
                Vnext = __shfl_sync(FULL, mine, (cnt - 1) / E);
                if (last_tau >= 0 && s2 >= cnt) Vnext = 0.0f;  // still reset / refractory
            }
            if (last_tau < 0)
                aw = df_mul(aw, pdf(cnt));
            else
                aw = df_mul(pdf(cnt - last_tau - 1), A1);
            Vin = Vnext;
            rel -= cnt;
        }
        if (dead) break;
        if (A.fin && lane == 0) {
            AlifState fs;
            fs.v = Vin;
            fs.a = aw.hi;
            fs.rem = rel > 0 ? rel : 0;
            A.fin[r] = fs;
        }
        ++n_rows;
        __syncwarp();  // the p^j table is rewritten for the next row
    }

    if (LOAD == 1) {  // never leave a copy in flight into this CTA's shared memory
        while (consumed < issued) {
            const int st = consumed % NSTAGE;
            if (!mbar_wait_bounded(&bars[st], (consumed / NSTAGE) & 1u)) {
                report_timeout(A.status);
                break;
            }
            ++consumed;
        }
    }
    if (lane == 0 && A.counters) {
        atomicAdd(&A.counters[0], n_exact);
        atomicAdd(&A.counters[1], n_exact_spk);
        atomicAdd(&A.counters[2], n_rows);
    }
}

// Event buckets of the input raster for the fused projection: one warp per (batch element b,
// 32-step word w).  Lane l (step 32 w + l) gathers, 32 inputs at a time, the bits of the inputs
// active at its step (a 32 x 32 bit transpose of the inputs' words), counts them, and after a warp
// scan writes the step's offset into the word's row (33 offsets: steps 0..32) and the active
// inputs in ascending order into the word's bucket of `cap` entries.  A word with more than `cap`
// events records ALIF_EUNSUPPORTED in the status word (its currents are then incomplete).
__global__ void ev_bucket_kernel(const uint32_t *S, long long B, long long Nin, long long nw, long long T, int cap,
                                 int *off, uint16_t *ent, int *status) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= B * nw) return;
    const long long b = gw / nw, w = gw - b * nw;
    const int ng = (int)((Nin + 31) / 32);  // <= 32
    const uint32_t tail = (w == nw - 1 && (T & 31)) ? ((1u << (T & 31)) - 1u) : 0xffffffffu;
    uint32_t m[32];
    int cnt = 0;
#pragma unroll
    for (int g = 0; g < 32; ++g) {
        m[g] = 0u;
        if (g < ng) {
            const long long j = (long long)g * 32 + lane;
            const uint32_t x = j < Nin ? (__ldg(S + (b * Nin + j) * nw + w) & tail) : 0u;
            m[g] = bits_transpose32(x, lane);  // lane l: inputs g*32 + c active at step l (bit c)
            cnt += __popc(m[g]);
        }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    int *op = off + gw * EV_ROW;
    op[lane] = incl - cnt;
    if (lane == 31) op[32] = total;
    if (total > cap && lane == 0 && status) atomicExch(status, ALIF_EUNSUPPORTED);
    uint16_t *ep = ent + gw * cap;
    int pos = incl - cnt;
#pragma unroll
    for (int g = 0; g < 32; ++g) {
        uint32_t x = m[g];
        while (x) {
            const int c = __ffs(x) - 1;
            x &= x - 1u;
            if (pos < cap) ep[pos] = (uint16_t)(g * 32 + c);
            ++pos;
        }
    }
}

}  // namespace fwd

// Workspace of the fused forward: event offsets, then the event buckets (256-byte aligned parts).
size_t alif_forward_fused_ws(long long B, long long Nin, long long T, int cap) {
    (void)Nin;
    const long long nw = (T + 31) / 32;
    const size_t off_b = ((size_t)(B * nw * fwd::EV_ROW) * 4 + 255) & ~(size_t)255;
    const size_t ent_b = ((size_t)(B * nw * cap) * 2 + 255) & ~(size_t)255;
    return off_b + ent_b;
}

static int g_sm_count_fused = 0;

// Fused projection + block forward: builds the event buckets, then runs the forward with the
// currents computed from them (and written to I).  I, ws 16-byte aligned; Nin <= 1024.
int launch_alif_forward_fused(long long B, long long Nin, long long N, long long T, const float *W,
                              const uint32_t *S, const float *bias, const AlifNeuron *nrn, const AlifState *init,
                              int cap, float *I, uint32_t *spikes, AlifState *ckpt, AlifState *fin, void *ws,
                              unsigned long long *counters, int *status, cudaStream_t stream) {
    using namespace fwd;
    const long long nw = (T + 31) / 32;
    int *off = static_cast<int *>(ws);
    const size_t off_b = ((size_t)(B * nw * EV_ROW) * 4 + 255) & ~(size_t)255;
    uint16_t *ent = reinterpret_cast<uint16_t *>(static_cast<unsigned char *>(ws) + off_b);
    {
        const long long threads = B * nw * 32;
        long long Sarg_B = B, Sarg_Nin = Nin, Sarg_nw = nw, Sarg_T = T;
        int capv = cap;
        void *args[] = {const_cast<uint32_t **>(&S), &Sarg_B, &Sarg_Nin, &Sarg_nw, &Sarg_T, &capv, &off, &ent, &status};
        const cudaError_t e = cudaLaunchKernel((const void *)ev_bucket_kernel, dim3((unsigned)((threads + 255) / 256)),
                                               dim3(256), args, 0, stream);
        if (e != cudaSuccess) return (int)e;
    }
    Args A;
    memset(&A, 0, sizeof A);
    A.rows = B * N;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + HALF - 1) / HALF;
    A.nwin = (T + Geo<8>::WIN - 1) / Geo<8>::WIN;
    A.I = I;
    A.nrn = nrn;
    A.init = init;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.fin = fin;
    A.counters = counters;
    A.status = status;
    A.W = W;
    A.bias = bias;
    A.ev_off = off;
    A.ev_ent = ent;
    A.Nin = Nin;
    A.nw_in = nw;
    A.ev_cap = cap;
    if (g_sm_count_fused == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count_fused, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count_fused <= 0) g_sm_count_fused = 1;
    }
    static int occ = 0;
    constexpr int smem = Geo<8>::SMEM_BYTES;
    const void *fn = (const void *)fwd_kernel<2, false, false, 8>;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, WARPS * 32, smem);
        occ = n > 0 ? n : 1;
    }
    const long long need = (A.rows + WARPS - 1) / WARPS;
    const long long capb = (long long)g_sm_count_fused * occ;
    const int grid = (int)(need < capb ? need : capb);
    if (grid <= 0) return 0;
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    void *args[] = {&tm, &A};
    return (int)cudaLaunchKernel(fn, dim3(grid), dim3(WARPS * 32), args, smem, stream);
}

// --------------------------------------------------------------- launcher
static int g_sm_count = 0;
static int g_fwd_window = 0;  // 0: chosen from the row count; 256 or 512: forced
static int g_fwd_layout = 0;  // 0: chosen from the row count; 1: a warp per row; 2: a lane per row

int launch_alif_forward_rows(long long rows, long long N, long long T, const float *I, const AlifNeuron *nrn,
                             const AlifState *init, uint32_t *spikes, AlifState *ckpt, AlifState *fin,
                             unsigned long long *counters, int *status, cudaStream_t stream, bool *declined);

template <int LOAD, bool VTR, bool ATR, int E>
static int launch_fwd(const CUtensorMap &tm, const fwd::Args &A, cudaStream_t stream) {
    using namespace fwd;
    constexpr int smem = Geo<E>::SMEM_BYTES;
    static int occ = 0;
    const void *fn = (const void *)fwd_kernel<LOAD, VTR, ATR, E>;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, WARPS * 32, smem);
        occ = n > 0 ? n : 1;
    }
    // one resident wave: CTAs per SM from the occupancy of the selected variant
    const long long need = (A.rows + WARPS - 1) / WARPS;
    const long long cap = (long long)g_sm_count * occ;
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return 0;
    // the launch's own status (cudaGetLastError could report an earlier, unrelated failure)
    void *args[] = {const_cast<CUtensorMap *>(&tm), const_cast<Args *>(&A)};
    return (int)cudaLaunchKernel(fn, dim3(grid), dim3(WARPS * 32), args, smem, stream);
}

int launch_alif_forward(long long B, long long N, long long T, const float *I,
                        const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                        float *vtr, float *atr, AlifState *ckpt, AlifState *fin,
                        unsigned long long *counters, int *status, cudaStream_t stream) {
    using namespace fwd;
    Args A;
    memset(&A, 0, sizeof A);
    A.rows = B * N;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + HALF - 1) / HALF;
    A.I = I;
    A.nrn = nrn;
    A.init = init;
    A.spikes = spikes;
    A.vtr = vtr;
    A.atr = atr;
    A.ckpt = ckpt;
    A.fin = fin;
    A.counters = counters;
    A.status = status;
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    // a lane per row when the rows alone fill every SM's warp slots several times over (traces
    // are written by the warp-per-row kernel); it declines calls it cannot stage with TMA
    const bool lanes = g_fwd_layout == 2 || (g_fwd_layout == 0 && A.rows >= 32LL * g_sm_count);
    if (lanes && !vtr && !atr) {
        bool declined = false;
        const int rc =
            launch_alif_forward_rows(A.rows, N, T, I, nrn, init, spikes, ckpt, fin, counters, status, stream, &declined);
        if (!declined) return rc;
    }
    auto aligned16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    // 2-D view of I as [rows * T / 16, 16] floats: T a multiple of 16, 16-byte aligned
    // base and traces, and box coordinates within int32.
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    bool tma = (T % 16 == 0) && aligned16(I) && (!vtr || aligned16(vtr)) && (!atr || aligned16(atr)) &&
               (A.rows * T / 16 + 32 < (1LL << 31));
    // 512-step windows when the rows leave warp slots empty (each row's chain of windows is then
    // the limit, and longer windows halve it), 256-step windows (four CTAs per SM) otherwise; the
    // wide kernel serves the TMA path without traces
    bool wide = g_fwd_window == 512 || (g_fwd_window == 0 && A.rows <= 8LL * g_sm_count);
    wide = wide && tma && !vtr && !atr;
    const long long win = wide ? Geo<16>::WIN : Geo<8>::WIN;
    if (tma && make_rows16_map(&tm, I, A.rows * T / 16, (unsigned)(win / 16)) != 0) {
        tma = false;
        wide = false;
        memset(&tm, 0, sizeof tm);
    }
    A.nwin = (T + (wide ? Geo<16>::WIN : Geo<8>::WIN) - 1) / (wide ? Geo<16>::WIN : Geo<8>::WIN);
    if (wide) return launch_fwd<1, false, false, 16>(tm, A, stream);
    switch ((tma ? 4 : 0) | (vtr ? 2 : 0) | (atr ? 1 : 0)) {
        case 0: return launch_fwd<0, false, false, 8>(tm, A, stream);
        case 1: return launch_fwd<0, false, true, 8>(tm, A, stream);
        case 2: return launch_fwd<0, true, false, 8>(tm, A, stream);
        case 3: return launch_fwd<0, true, true, 8>(tm, A, stream);
        case 4: return launch_fwd<1, false, false, 8>(tm, A, stream);
        case 5: return launch_fwd<1, false, true, 8>(tm, A, stream);
        case 6: return launch_fwd<1, true, false, 8>(tm, A, stream);
        default: return launch_fwd<1, true, true, 8>(tm, A, stream);
    }
}

}  // namespace alif

// Window length of the block forward (see include/alif.h).
extern "C" int alif_forward_window(int steps) {
    if (steps != 0 && steps != 256 && steps != 512) return ALIF_EINVAL;
    const int prev = alif::g_fwd_window;
    alif::g_fwd_window = steps;
    return prev;
}

// Layout of the block forward (see include/alif.h).
extern "C" int alif_forward_layout(int layout) {
    if (layout < 0 || layout > 2) return ALIF_EINVAL;
    const int prev = alif::g_fwd_layout;
    alif::g_fwd_layout = layout;
    return prev;
}
