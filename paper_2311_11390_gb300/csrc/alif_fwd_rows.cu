// ARP-blocked ALIF forward with one neuron row per lane (Section 3, Props 1-5) for sm_103a.
//
// With many rows (B N well above the SM count) the rows alone fill the GPU, and the time
// parallelism inside a row that the warp-per-row kernel spends a warp on is not needed.  This
// kernel gives each lane one row and walks it through Blocks of K steps, K <= T_R, so that a
// Block holds at most one spike (Section 3.1); a Block's steps are independent operations inside
// the lane:
//   1. the no-reset membrane of Prop 1 from the state entering the Block,
//        V~[k] = beta^{k+1} v_in + L[k],   L[k] = sum_{j<=k} beta^{k-j} m[j] c I[j],
//      where L depends on the inputs only (a K-step chain) and the beta^{k+1} are FP64-derived
//      powers rounded once;
//   2. the threshold theta0 + d p^k a_in (Prop 5: no spike yet inside the Block);
//   3. the first crossing V~ > theta (Eqs 7-9: the Block's later faulty spikes are discarded);
//   4. the state entering the next Block (Props 4 and 5): after a spike at k the membrane is 0,
//      the rest of the Block lies in the refractory span (K <= T_R) and a = p^{K-1-k} (p a_k + 1);
//      otherwise v = V~[K-1] and a = p^K a_in.
// A warp holds 32 consecutive rows.  K = 16 when every row of the warp has T_eff >= 16, else 8, 4
// or 2 (T_eff >= 2 always).  The state chain of a row costs O(1) dependent operations per Block, the
// sequential depth of the method; the L chains run ahead of it.
//
// Input: stages of [32 rows x 64 steps] (two 2-D TMA boxes of 32 x 32 floats, 128-byte swizzle)
// in a three-deep ring per warp; a lane reads its own row's K steps with 16-byte loads, which
// the swizzle spreads over distinct bank groups.
//
// Exactness of the spike decisions, as in the warp-per-row kernel: the FP32 margin comes with an
// error bound G, and a margin within G is re-decided in double-single arithmetic from the lane's
// exact anchor (the last reset, where V is 0, or the last re-decided step), warp-cooperatively,
// one ambiguous lane at a time.  The carried membrane is double-single, so a Block's FP32
// rounding does not accumulate from Block to Block.  With u = 2^-24, the margin of step k errs by
// at most the sum of
//  - the Block's input chain: L[k] (rounded c and beta, one rounding of c I[j], one per FMA) errs by
//    at most (2k + 2) u of sum_j beta^(k-j) c |I[j]| <= (1 - beta^(k+1)) R max_Block|I|; a Block
//    entered with the effective membrane adds the error of L[r-1] and the three roundings of
//    W's factor and product: at most (4K + 2) u R (1 - beta^K) max_Block|I| in all;
//  - the carried membrane's error: each Block adds at most (2K + 1) u R (1 - beta^K) max_Block|I|
//    (its chain's end, refractory entries included) and the sum decays by beta^K per Block, so it
//    stays below (2K + 1) u R max_row|I|; a reset clears it;
//  - the local roundings: v_in's rounded power and dropped low part (2 u |v_in|), the membrane's FMA
//    (u |V~|), d a's three roundings (3 u |d a|), the margin's FMA (u |Z|) and theta0 - G (u theta0).
// With |V~| <= M = max(|v_in|, R max_Block|I|) and |Z| <= M + |d a|, G is
//   (1 + 2^-6) (u (4 M + 5 |d a| + theta0) + (4K + 4) u R (1 - beta^K) max_Block|I| + (2K + 4) u R max_row|I|),
// the slack covering the double-single carries' second-order terms and G's own FP32 evaluation.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "exact_membrane.cuh"
#include "tmap.h"

namespace alif {
namespace fwdr {

#ifndef ALIF_ROWS_SPAN
#define ALIF_ROWS_SPAN 64  // steps per stage (a multiple of 32: one box per 32 steps)
#endif
#ifndef ALIF_ROWS_NST
#define ALIF_ROWS_NST 3  // stages per warp
#endif
constexpr int SPAN = ALIF_ROWS_SPAN;
constexpr int NST = ALIF_ROWS_NST;
constexpr int NBOX = SPAN / 32;                // boxes per stage
constexpr int BOX_BYTES = 32 * 32 * 4;         // 32 rows x 32 steps
constexpr int STAGE_BYTES = NBOX * BOX_BYTES;  // 8 KB
static_assert(SPAN % 32 == 0 && NBOX >= 1, "stages of whole boxes");
constexpr int KMAX = 16;                       // longest Block
// the ring, its barriers, the lanes' p^k tables (float2 [KMAX][32]) and beta^-r tables (float
// [KMAX][32]), alignment of the swizzled ring
constexpr int SMEM_BYTES = NST * STAGE_BYTES + NST * 8 + KMAX * 32 * 12 + 1024;

struct Args {
    long long rows, N, T, nwords, nckpt, ngroups;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    uint32_t *spikes;
    AlifState *ckpt, *fin;
    unsigned long long *counters;  // [0] re-decided margins, [1] of which spikes, [2] rows
    int *status;
};

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

template <int K>
__device__ __forceinline__ float vmaxk(const float (&v)[K]) {
    if constexpr (K == 2) return fmaxf(v[0], v[1]);
    else if constexpr (K == 4) return max3f(v[0], v[1], fmaxf(v[2], v[3]));
    else if constexpr (K == 8) return max3f(max3f(v[0], v[1], v[2]), max3f(v[3], v[4], v[5]), fmaxf(v[6], v[7]));
    else
        return max3f(max3f(max3f(v[0], v[1], v[2]), max3f(v[3], v[4], v[5]), max3f(v[6], v[7], v[8])),
                     max3f(v[9], v[10], v[11]), max3f(max3f(v[12], v[13], v[14]), v[15], v[15]));
}

template <int K>
__device__ __forceinline__ float absmaxk(const float (&v)[K]) {
    float a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = fabsf(v[k]);
    return vmaxk<K>(a);
}

// v[k] by a select tree on the bits of k (0 <= k < K).
template <int K>
__device__ __forceinline__ float pickk(const float (&v)[K], int k) {
    float a[K / 2];
#pragma unroll
    for (int i = 0; i < K / 2; ++i) a[i] = (k & 1) ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int w = K / 4, bit = 2; w >= 1; w /= 2, bit *= 2) {
#pragma unroll
        for (int i = 0; i < w; ++i) a[i] = (k & bit) ? a[2 * i + 1] : a[2 * i];
    }
    return a[0];
}

// a * b + c for double-single a, b and a float c.
__device__ __forceinline__ df df_fma_f(df a, df b, float c) {
    df p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    df s = two_sum(p.hi, c);
    s.lo = __fadd_rn(s.lo, p.lo);
    return quick_two_sum(s.hi, s.lo);
}

// a + b for double-single a, b with one TwoSum on the high parts (absolute error ~u^2 (|a| + |b|)).
__device__ __forceinline__ df df_add_sloppy(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, s.lo);
}

__global__ void __launch_bounds__(32) fwd_rows_kernel(const __grid_constant__ CUtensorMap tm, const Args A) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 128-byte swizzle: 1024-aligned boxes
    float *ring = reinterpret_cast<float *>(sm);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NST * STAGE_BYTES);
    // p^k, k < K, of each lane's row as double-single pairs at [k][lane] (dynamic-index lookups)
    float2 *ptab = reinterpret_cast<float2 *>(sm + NST * STAGE_BYTES + NST * 8);
    // beta^-r, 0 < r < K, of each lane's row at [r][lane]
    float *btab = reinterpret_cast<float *>(ptab + KMAX * 32);
    const int lane = threadIdx.x;
    const long long ng = gridDim.x;
    if ((long long)blockIdx.x >= A.ngroups) return;
    const int nstg = (int)((A.T + SPAN - 1) / SPAN);

    // ---- TMA producer (lane 0 issues; every lane tracks the cursor): stages of each group in
    // order, groups g, g + gridDim.x, ...
    long long p_g = blockIdx.x;
    int p_s = 0;
    unsigned issued = 0, consumed = 0;
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&]() {
        while (p_g < A.ngroups && issued - consumed < (unsigned)NST) {
            if (lane == 0) {
                const int st = issued % NST;
                const uint32_t dst = smem_u32(ring) + st * STAGE_BYTES, bar = smem_u32(&bars[st]);
                const int x = p_s * SPAN, y = (int)(p_g * 32);
                // boxes holding steps < T only (no box lies wholly outside the tensor)
                const long long left = A.T - x;
                const int nbx = left >= SPAN ? NBOX : (int)((left + 31) / 32);
                mbar_arrive_expect_tx(&bars[st], nbx * BOX_BYTES);
                for (int b = 0; b < nbx; ++b) tma_load_2d_u(dst + b * BOX_BYTES, &tm, x + 32 * b, y, bar);
            }
            ++issued;
            if (++p_s == nstg) {
                p_s = 0;
                p_g += ng;
            }
        }
    };
    issue();

    const int sw = lane & 7;  // this lane's row in the swizzle pattern
    unsigned n_exact = 0, n_exact_spk = 0, n_rows = 0;
    bool dead = false;
    for (long long g = blockIdx.x; g < A.ngroups && !dead; g += ng) {
        const long long r = g * 32 + lane;
        const bool live = r < A.rows;
        const AlifNeuron nr = A.nrn[(live ? r : g * 32) % A.N];
        const int tmin = (int)__reduce_min_sync(FULL, live ? (unsigned)nr.teff : 0x7fffffffu);

        // One group of 32 rows with K-step Blocks; false if a stage never arrived.
        auto group = [&](auto ktag) -> bool {
            constexpr int K = decltype(ktag)::value;
            static_assert(K <= KMAX && SPAN % K == 0, "Blocks tile the stages and fit the lane tables");
            const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
            const float bf = nr.beta_hi, c = nr.c_hi, d = nr.d, th0 = nr.theta0, Rr = nr.R;
            const int teff = nr.teff;
            float Bk[K];  // beta^(k+1)
            float Ph[K];  // p^k (the double-single pairs are in the lane's column of ptab)
            df BK, PK;    // beta^K, p^K
            {
                df q{1.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    q = df_mul(q, beta);
                    Bk[k] = q.hi;
                }
                BK = q;
                df s{1.0f, 0.0f};
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    Ph[k] = s.hi;
                    ptab[k * 32 + lane] = make_float2(s.hi, s.lo);
                    s = df_mul(s, p);
                }
                PK = s;
                df q2{1.0f, 0.0f};
#pragma unroll
                for (int k = 1; k < K; ++k) {
                    q2 = df_mul(q2, beta);
                    btab[k * 32 + lane] = 1.0f / q2.hi;
                }
            }
            // A lane whose Block starts with r (0 < r < K) refractory steps enters it with the
            // effective membrane W = -beta^-r L[r-1] (the unmasked input chain): V~[k] = beta^{k+1} W
            // + L[k] = sum_{r<=j<=k} beta^{k-j} c I[j] for k >= r, the masked membrane, at the cost of
            // one lookup.  Rows whose beta^K leaves the normal range recompute the masked chain.
            const bool weff = __all_sync(FULL, !live || BK.hi >= 7.9e-31f);  // beta^K >= 2^-100
            __syncwarp();
            // error bound (header) G = gV max(|v_in|, R max_Block|I|) + gD |d a| + gA max_Block|I|
            // + gB max_row|I| + g0, each factor with the 1 + 2^-6 slack; u = 2^-24
            constexpr float u = 5.9604645e-8f, us = u * 1.015625f;
            const float omb = fmaxf((1.0f - BK.hi) - BK.lo, 0.0f);  // 1 - beta^K bounds a Block's L / (R max|I|)
            const float gV = 4.0f * us, gD = 5.0f * us, g0 = us * th0, gA = (4.0f * K + 4.0f) * us * Rr * omb,
                        gB = (2.0f * K + 4.0f) * us * Rr;
            const int T = (int)A.T;

            // ---- state entering the row
            AlifState s0{0.0f, 0.0f, 0};
            if (A.init && live) s0 = A.init[r];
            int rel = s0.rem > 0 ? s0.rem : 0;   // steps still masked (refractory) from the Block start
            df Vd{rel > 0 ? 0.0f : s0.v, 0.0f};  // membrane entering the Block
            df aw{s0.a, 0.0f};                   // adaptation entering the Block
            int anc_t = rel;                     // exact anchor: V entering step anc_t is anc_v
            df anc_v = Vd;
            float mxr = 0.0f;  // running max |I| of the row
            uint32_t sword = 0;
            AlifState *ck = (A.ckpt && live) ? A.ckpt + r * A.nckpt : nullptr;
            uint32_t *spw = A.spikes + (live ? r : 0) * A.nwords;

            // ---- staging: the stage holding the current word; a lane's K inputs of a Block
            const float *stg = nullptr;  // this lane's box row in that stage
            auto wait_stage = [&]() -> bool {
                const int st = consumed % NST;
                if (!mbar_wait_bounded(&bars[st], (consumed / NST) & 1u)) {
                    report_timeout(A.status);
                    return false;
                }
                stg = ring + st * (STAGE_BYTES / 4) + lane * 32;
                return true;
            };
            auto release_stage = [&]() {  // the stage's inputs are all in registers
                __syncwarp();
                fence_proxy_async_smem();
                ++consumed;
                issue();
            };
            auto checkpoint = [&](int t) {  // the state entering step t (a multiple of 256)
                if (ck) {
                    AlifState cs;
                    cs.v = Vd.hi;
                    cs.a = aw.hi;
                    cs.rem = rel;
                    ck[t / ALIF_CKPT_STEPS] = cs;
                }
            };

            // One Block: steps tb .. tb + cnt - 1 (cnt = K unless FULLB is false), inputs from step o of
            // the stage.
            auto block = [&](auto fulltag, int tb, int o, int cnt_in) {
                constexpr bool FULLB = decltype(fulltag)::value;
                const int cnt = FULLB ? K : cnt_in;
                float x[K];
                {
                    const float *bx = stg + (o >> 5) * 1024;
                    const int w = o & 31;
                    if constexpr (K >= 4) {
#pragma unroll
                        for (int q = 0; q < K / 4; ++q) {
                            const float4 u = *reinterpret_cast<const float4 *>(bx + 4 * (((w >> 2) + q) ^ sw));
                            x[4 * q] = u.x;
                            x[4 * q + 1] = u.y;
                            x[4 * q + 2] = u.z;
                            x[4 * q + 3] = u.w;
                        }
                    } else {
                        const float2 u = *reinterpret_cast<const float2 *>(bx + 4 * ((w >> 2) ^ sw) + (w & 3));
                        x[0] = u.x;
                        x[1] = u.y;
                    }
                }

                // ---- 1. no-reset membrane.  L[k] = sum_{j<=k} beta^{k-j} c I[j] (no mask); a lane
                // whose Block starts with r refractory steps (0 < r < K) enters with the effective
                // membrane W = -beta^-r L[r-1], so that V~[k] = beta^{k+1} W + L[k] is the masked
                // membrane for k >= r (Eq 4); rows whose beta^K leaves the normal range recompute the
                // masked chain instead.  The Block's masked steps are no candidates.
                float L[K];
                {
                    float cx[K];
                    const float2 cc = make_float2(c, c);
#pragma unroll
                    for (int i = 0; i < K / 2; ++i) {
                        const float2 v = __fmul2_rn(cc, make_float2(x[2 * i], x[2 * i + 1]));
                        cx[2 * i] = v.x;
                        cx[2 * i + 1] = v.y;
                    }
                    if (!weff && __any_sync(FULL, rel > 0)) {
#pragma unroll
                        for (int k = 0; k < K; ++k) cx[k] = k >= rel ? cx[k] : 0.0f;
                    }
                    L[0] = cx[0];
#pragma unroll
                    for (int k = 1; k < K; ++k) L[k] = fmaf(bf, L[k - 1], cx[k]);
                }
                float vin = Vd.hi;
                if (weff && rel > 0 && rel < K)  // (per lane: skipped unless a lane of the warp needs it)
                    vin = -pickk<K>(L, rel - 1) * btab[rel * 32 + lane];
                float V[K], Z[K];  // V~ and the margins Z = V~ - d p^k a_in
                const float dA = d * aw.hi;
                {
                    const float2 vv = make_float2(vin, vin), nd = make_float2(-dA, -dA);
#pragma unroll
                    for (int i = 0; i < K / 2; ++i) {
                        const float2 v =
                            __ffma2_rn(make_float2(Bk[2 * i], Bk[2 * i + 1]), vv, make_float2(L[2 * i], L[2 * i + 1]));
                        const float2 z = __ffma2_rn(nd, make_float2(Ph[2 * i], Ph[2 * i + 1]), v);
                        V[2 * i] = v.x;
                        V[2 * i + 1] = v.y;
                        Z[2 * i] = z.x;
                        Z[2 * i + 1] = z.y;
                    }
                }
                // the carries without a spike (they do not wait for the crossing search below)
                df Vn, an;
                const df vind{vin, rel > 0 ? 0.0f : Vd.lo};
                if (FULLB) {
                    Vn = df_fma_f(BK, vind, L[K - 1]);
                    an = df_mul(aw, PK);
                } else {
                    Vn = df_fma_f(df_pow(beta, cnt), vind, pickk<K>(L, cnt - 1));
                    const float2 pc = ptab[(cnt & (K - 1)) * 32 + lane];  // cnt < K here unless cnt == K
                    an = cnt == K ? df_mul(aw, PK) : df_mul(aw, df{pc.x, pc.y});
                }
                // ---- 2.-3. error bound and first crossing: usually no lane comes near theta
                const float mx = absmaxk<K>(x);  // steps past T read as 0
                mxr = fmaxf(mxr, mx);
                // |V~| <= max(|v_in|, R max|I|) (v_in = 0 for a refractory lane)
                const float G =
                    fmaf(gV, fmaxf(rel > 0 ? 0.0f : fabsf(vin), Rr * mx), fmaf(gD, fabsf(dA), fmaf(gA, mx, fmaf(gB, mxr, g0))));
                const float thr = th0 - G;  // a candidate where Z >= thr
                unsigned zb = 0u;
                if (__any_sync(FULL, live && rel < K && vmaxk<K>(Z) >= thr)) {
                    if (live) {
#pragma unroll
                        for (int k = 0; k < K; ++k)
                            if (Z[k] >= thr) zb |= 1u << k;
                        zb &= ((1u << cnt) - 1u) & ~((1u << (rel < K ? rel : K)) - 1u);  // admitted steps
                    }
                    // re-decide margins inside the error band exactly, lane by lane, until every
                    // lane's first remaining candidate is a sure spike (or it has none)
                    bool sure = false;
                    while (true) {
                        const int myk = __ffs(zb) - 1;
                        bool amb = false;
                        if (zb != 0u && !sure) amb = !(pickk<K>(Z, myk & (K - 1)) - thr > 2.0f * G);
                        unsigned am = __ballot_sync(FULL, amb);
                        if (am == 0u) break;
                        do {
                            const int Lx = __ffs(am) - 1;
                            am &= am - 1u;
                            const int kx = __shfl_sync(FULL, myk, Lx);
                            const int at = __shfl_sync(FULL, anc_t, Lx);
                            const float avh = __shfl_sync(FULL, anc_v.hi, Lx), avl = __shfl_sync(FULL, anc_v.lo, Lx);
                            const float bh = __shfl_sync(FULL, nr.beta_hi, Lx), bl = __shfl_sync(FULL, nr.beta_lo, Lx);
                            const float ch = __shfl_sync(FULL, nr.c_hi, Lx), cl = __shfl_sync(FULL, nr.c_lo, Lx);
                            df thx{0.0f, 0.0f};
                            if (lane == Lx) {  // theta = theta0 + d a_in p^k, double-single
                                const float2 pk = ptab[kx * 32 + lane];
                                thx = df_add(df_mul_f(df_mul(aw, df{pk.x, pk.y}), d), df{th0, 0.0f});
                            }
                            thx.hi = __shfl_sync(FULL, thx.hi, Lx);
                            thx.lo = __shfl_sync(FULL, thx.lo, Lx);
                            const int tg = tb + kx;
                            const df Vx = exact_membrane<false>(A.I + (g * 32 + Lx) * A.T, at, avh, avl, tg, bh, bl,
                                                                ch, cl, lane);
                            if (lane == Lx) {
                                ++n_exact;
                                if (df_cmp(Vx, thx) <= 0) {
                                    anc_t = tg + 1;  // exact V is now known entering tg + 1
                                    anc_v = Vx;
                                    zb &= ~((2u << kx) - 1u);
                                } else {
                                    ++n_exact_spk;
                                    sure = true;
                                }
                            }
                        } while (am);
                    }
                }

                // ---- 4. the state entering the next Block (Props 3-5).  After a spike at kc the
                // membrane is 0, the rest of the Block is refractory (K <= T_eff) and
                // a = p^cnt a_in + p^(cnt-1-kc) (the spike's unit, decayed); a wholly refractory
                // Block ends at 0; otherwise the carry beta^cnt v_in + L[cnt-1] (double-single).
                const bool spk = zb != 0u;
                const int kc = __ffs(zb) - 1;
                const float2 pm = ptab[(spk ? cnt - 1 - kc : 0) * 32 + lane];
                aw = df_add_sloppy(an, spk ? df{pm.x, pm.y} : df{0.0f, 0.0f});
                Vd = (spk || rel >= cnt) ? df{0.0f, 0.0f} : Vn;
                rel = spk ? kc + teff - cnt : (rel > cnt ? rel - cnt : 0);  // kc + teff - cnt >= 0: K <= T_eff
                anc_t = spk ? tb + kc + teff : anc_t;  // V is exactly 0 entering the first admitted step
                anc_v = spk ? df{0.0f, 0.0f} : anc_v;
                sword |= spk ? 1u << ((tb & 31) + kc) : 0u;
            };

            // ---- the row: full 32-step words (two per stage, a spike word each, a checkpoint every
            // eighth), then the last, partial word (T % 32 steps)
            constexpr int WPS = SPAN / 32;  // words per stage
            constexpr int BPW = 32 / K;     // Blocks per word
            const int nfw = T >> 5;
            if (!wait_stage()) return false;
            for (int wd = 0; wd < nfw; ++wd) {
                if (wd > 0 && (wd & (WPS - 1)) == 0) {  // the word opens the next stage
                    release_stage();
                    if (!wait_stage()) return false;
                }
                if ((wd & 7) == 0) checkpoint(wd << 5);
                const int ow = (wd & (WPS - 1)) << 5;  // the word's first step within the stage
                if constexpr (K >= 8) {
#pragma unroll
                    for (int j = 0; j < BPW; ++j) block(std::true_type{}, (wd << 5) + j * K, ow + j * K, K);
                } else {
#pragma unroll 1
                    for (int j = 0; j < BPW; ++j) block(std::true_type{}, (wd << 5) + j * K, ow + j * K, K);
                }
                if (live) spw[wd] = sword;
                sword = 0;
            }
            const int tt = nfw << 5;
            if (tt < T) {
                if (nfw > 0 && (nfw & (WPS - 1)) == 0) {
                    release_stage();
                    if (!wait_stage()) return false;
                }
                if ((nfw & 7) == 0) checkpoint(tt);
                const int ow = (nfw & (WPS - 1)) << 5;
#pragma unroll 1
                for (int tb = tt; tb < T; tb += K) block(std::false_type{}, tb, ow + (tb - tt), T - tb >= K ? K : T - tb);
                if (live) spw[nfw] = sword;
                sword = 0;
            }
            release_stage();  // the row's last stage
            if (A.fin && live) {
                AlifState fs;
                fs.v = Vd.hi;
                fs.a = aw.hi;
                fs.rem = rel;
                A.fin[r] = fs;
            }
            return true;
        };
        bool ok;
        if (tmin >= 16)
            ok = group(std::integral_constant<int, 16>{});
        else if (tmin >= 8)
            ok = group(std::integral_constant<int, 8>{});
        else if (tmin >= 4)
            ok = group(std::integral_constant<int, 4>{});
        else
            ok = group(std::integral_constant<int, 2>{});
        dead = !ok;
        if (live) ++n_rows;
    }

    // never leave a copy in flight into this CTA's shared memory
    while (consumed < issued) {
        if (!mbar_wait_bounded(&bars[consumed % NST], (consumed / NST) & 1u)) {
            report_timeout(A.status);
            break;
        }
        ++consumed;
    }
    n_exact = __reduce_add_sync(FULL, n_exact);
    n_exact_spk = __reduce_add_sync(FULL, n_exact_spk);
    n_rows = __reduce_add_sync(FULL, n_rows);
    if (lane == 0 && A.counters) {
        atomicAdd(&A.counters[0], n_exact);
        atomicAdd(&A.counters[1], n_exact_spk);
        atomicAdd(&A.counters[2], n_rows);
    }
}

}  // namespace fwdr

static int g_sm_count_rows = 0;

// Row-per-lane forward: the launch's status.  *declined is set (nothing launched) when the input
// cannot be staged with TMA (T % 4 != 0, I not 16-byte aligned, or the tensor map is rejected);
// the caller then uses the warp-per-row kernel.
int launch_alif_forward_rows(long long rows, long long N, long long T, const float *I, const AlifNeuron *nrn,
                             const AlifState *init, uint32_t *spikes, AlifState *ckpt, AlifState *fin,
                             unsigned long long *counters, int *status, cudaStream_t stream, bool *declined) {
    using namespace fwdr;
    *declined = true;
    // step indices (plus a refractory span of at most 1e6 steps) stay within int32
    if (T % 4 != 0 || ((uintptr_t)I & 15u) != 0 || T >= (1LL << 30) || rows >= (1LL << 31)) return 0;
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    if (make_rowmajor_map(&tm, I, rows, T) != 0) return 0;
    *declined = false;
    Args A;
    memset(&A, 0, sizeof A);
    A.rows = rows;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS;
    A.ngroups = (rows + 31) / 32;
    A.I = I;
    A.nrn = nrn;
    A.init = init;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.fin = fin;
    A.counters = counters;
    A.status = status;
    if (g_sm_count_rows == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count_rows, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count_rows <= 0) g_sm_count_rows = 1;
    }
    static int occ = 0;
    const void *fn = (const void *)fwd_rows_kernel;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32, SMEM_BYTES);
        occ = n > 0 ? n : 1;
    }
    const long long cap = (long long)g_sm_count_rows * occ;
    const int grid = (int)(A.ngroups < cap ? A.ngroups : cap);
    if (grid <= 0) return 0;
    void *args[] = {&tm, &A};
    return (int)cudaLaunchKernel(fn, dim3(grid), dim3(32), args, SMEM_BYTES, stream);
}

}  // namespace alif
