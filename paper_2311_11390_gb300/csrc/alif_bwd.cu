// Surrogate-gradient backward of the blocked ALIF forward (sm_103a).
//
// Gradients are "detached" (Supplementary, "Detaching gradients"): S[t-1] is a
// constant in the reset of Eq 2 and in the adaptation update of Eq 5, and the
// ARP mask of Eq 4 carries no gradient; dS/dV is the fast-sigmoid surrogate
// 1/(k|V - theta| + 1)^2 (Supplementary, "Surrogate gradient"), reaching theta
// as -dS/du.  The reverse recurrences are linear:
//     G_V[t] = sg[t] gS[t] + gV[t] + beta (1 - S[t]) G_V[t+1]
//     G_a[t] = ga[t] - d sg[t] gS[t] + p G_a[t+1]
//     dL/dI[t] = (1 - beta) R m[t] G_V[t]
// One warp owns a row and walks its windows of 32 E steps from the last to the
// first (lane L holds steps E L .. E L + E - 1).  For each window it recomputes V
// and a from the checkpoint saved by the forward at the window start and the
// stored spike bits -- no spike decision is re-taken -- then runs both reverse
// recurrences as warp scans and accumulates the parameter gradients.  Windows
// without spikes or refractory carry-in take a lean path (plain decayed scans);
// the others use segmented scans whose factors are zero at the resets.
// Inputs are staged by 2-D TMA boxes (rows of 16 floats, 64-byte swizzle) into
// a per-warp ring, newest window first, when T is a multiple of 16; otherwise
// lanes read global memory directly.  E = 8 (256-step windows, one checkpoint
// stride) keeps the window's register arrays small enough for four CTAs of four
// warps per SM: the kernel is bound by the latency of its scan chains, and the
// warps hide it.  E = 16 (512-step windows, two CTAs per SM) serves calls whose
// rows leave warp slots empty, where each row's chain of windows sets the time.
// Per-row partial parameter sums go to the workspace; a second kernel sums them
// over the batch in a fixed order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "bwd_scan.cuh"
#include "common.cuh"
#include "tmap.h"

namespace alif {
namespace bwd {

#ifndef ALIF_BWD_MIN_BLOCKS
#define ALIF_BWD_MIN_BLOCKS 4
#endif
// Window geometry for E steps per lane: E = 8, 256-step windows (one checkpoint stride), sized for
// four CTAs of four warps per SM; E = 16, 512-step windows (two strides), two CTAs per SM.
template <int E>
struct Geo {
    static_assert(E == 8 || E == 16, "8 or 16 steps per lane");
    static constexpr int WIN = 32 * E;
    static constexpr int BOX = WIN * 4;               // one array's window
    static constexpr int CK = WIN / ALIF_CKPT_STEPS;  // checkpoint strides per window
    static constexpr int FOLD = 4096 / WIN;           // windows per double-single fold of the sums
    static constexpr int H = E / 2;                   // half-lane chain length
    static constexpr unsigned FULLM = (1u << E) - 1u, LOM = (1u << H) - 1u, HIM = FULLM & ~LOM;
    static constexpr int MIN_BLOCKS = E == 8 ? ALIF_BWD_MIN_BLOCKS : 2;
};
// TMA ring depth per warp.  Without trace gradients a window's stage is freed as soon as the
// lanes hold I and dL/dS in registers, so one stage already overlaps the next window's load with
// this window's compute (and the smaller shared-memory carve-out leaves more L1); with trace
// gradients the stage is read until the window ends, and a second stage keeps that overlap.
#ifndef ALIF_BWD_LEAN_STAGES
#define ALIF_BWD_LEAN_STAGES 1
#endif
template <bool GV, bool GA>
struct Ring {
    static constexpr int n = (GV || GA) ? 2 : ALIF_BWD_LEAN_STAGES;
};
constexpr int WARPS = 4;

struct Args {
    long long rows, N, T, nwords, nckpt, nwin;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    const uint32_t *spikes;
    const AlifState *ckpt;
    const float *gS, *gV, *ga, *gfin;
    float slope;
    float *gI, *ginit, *part;
    int *status;
};

template <bool GV, bool GA>
struct Narr {
    static constexpr int n = 2 + (GV ? 1 : 0) + (GA ? 1 : 0);
};

template <bool GV, bool GA, int E>
constexpr int smem_bytes() {
    return WARPS * Ring<GV, GA>::n * Narr<GV, GA>::n * Geo<E>::BOX + WARPS * Ring<GV, GA>::n * 8 +
           WARPS * 10 * 32 * 4 + 1024;
}

// LOAD: 1 = 2-D TMA ring, 0 = direct global loads; E steps per lane (Geo)
template <int LOAD, bool GV, bool GA, int SG, int E>
__global__ void __launch_bounds__(WARPS * 32, Geo<E>::MIN_BLOCKS)
    bwd_kernel(const __grid_constant__ CUtensorMap tmI, const __grid_constant__ CUtensorMap tmS,
               const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmA, const Args A) {
    constexpr int WIN = Geo<E>::WIN, BOX = Geo<E>::BOX, H = Geo<E>::H;
    // the beta sum in the same-step form (fast sigmoid, no trace gradients, TMA staging: the variants
    // the follow-up kernel can complete)
    constexpr bool SAMESTEP = SG == 0 && !GV && !GA && LOAD == 1;
    constexpr unsigned FULLM = Geo<E>::FULLM, LOM = Geo<E>::LOM, HIM = Geo<E>::HIM;
    constexpr int NARR = Narr<GV, GA>::n;
    constexpr int NSTAGE = Ring<GV, GA>::n;
    constexpr int STAGE = NARR * WIN;  // floats per stage
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(sm) + (size_t)warp * NSTAGE * STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + WARPS * NSTAGE * NARR * BOX) + warp * NSTAGE;
    // the lane's double-single parameter sums (hi of sum q at [q][lane], lo at [5 + q][lane]), kept in
    // shared memory rather than registers: they change only every 4096 steps
    float *accs =
        reinterpret_cast<float *>(sm + WARPS * NSTAGE * NARR * BOX + WARPS * NSTAGE * 8) + warp * 10 * 32 + lane;
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long nw = (long long)gridDim.x * WARPS;
    if (gw >= A.rows) return;

    // ---- producer: windows newest first, rows in order
    long long p_row = gw;
    int p_wi = (int)A.nwin - 1;
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
                const uint32_t dst = smem_u32(ring + st * STAGE), bar = smem_u32(&bars[st]);
                const int y = (int)((p_row * A.T + (long long)p_wi * WIN) >> 4);
                mbar_arrive_expect_tx(&bars[st], NARR * BOX);
                tma_load_2d_u(dst, &tmI, 0, y, bar);
                tma_load_2d_u(dst + BOX, &tmS, 0, y, bar);
                if (GV) tma_load_2d_u(dst + 2 * BOX, &tmV, 0, y, bar);
                if (GA) tma_load_2d_u(dst + (GV ? 3 : 2) * BOX, &tmA, 0, y, bar);
            }
            ++issued;
            if (--p_wi < 0) {
                p_wi = (int)A.nwin - 1;
                p_row += nw;
            }
        }
    };
    if (LOAD == 1) issue();

    const int t0 = E * lane;
    // this lane's E floats in a stage: 16-byte chunks ch0 .. ch0 + E/4 - 1 of box row t0 / 16, under the
    // 64-byte swizzle of that row (a quarter warp's 16-byte reads fall in distinct bank groups)
    const int swz = ((t0 >> 4) >> 1) & 3, ch0 = (t0 & 15) >> 2, brow = 16 * (t0 >> 4);
    bool dead = false;
    for (long long r = gw; r < A.rows && !dead; r += nw) {
        const AlifNeuron nr = A.nrn[r % A.N];
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        const float bf = beta.hi, pf = p.hi, c = nr.c_hi, d = nr.d, th0 = nr.theta0;
        const int teff = nr.teff;
        float Bb[5], Bp[5];  // decays of spans of 2^l lanes: beta^(E 2^l), p^(E 2^l)
        // anchors of the decay of the window-entry adaptation at the lane's steps 0 and H (the
        // products after them are FP32 chains of at most H - 1 steps): p^{t0}, p^{t0+H}; and the
        // half-lane decays beta^H, p^H.  The entering membrane joins the scans as beta vin added
        // to the window's first input.
        float Pa0, Pa4, b4f, p4f;
        {
            {
                const df b4 = df_pow(beta, H), pa = df_pow(p, t0), p4 = df_pow(p, H);
                Pa0 = pa.hi;
                Pa4 = df_mul(pa, p4).hi;
                b4f = b4.hi;
                p4f = p4.hi;
            }
            df b8 = df_pow(beta, E), p8 = df_pow(p, E);
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                Bb[l] = b8.hi;
                Bp[l] = p8.hi;
                b8 = df_mul(b8, b8);
                p8 = df_mul(p8, p8);
            }
        }
        const uint32_t *bits = A.spikes + r * A.nwords;

        auto load_state = [&](int wi) {
            AlifState st{0.0f, 0.0f, 0};
            if (A.ckpt)
                st = A.ckpt[r * A.nckpt + (long long)Geo<E>::CK * wi];
            else if (A.init)
                st = A.init[r];
            return st;
        };
        auto load_word = [&](int wi) {
            const long long widx = (long long)wi * (WIN / 32) + (t0 >> 5);
            return widx < A.nwords ? __ldg(bits + widx) : 0u;
        };
        AlifState cs_next = load_state((int)A.nwin - 1);
        uint32_t wd_next = load_word((int)A.nwin - 1);

        float gcV = A.gfin ? A.gfin[2 * r] : 0.0f;      // dL/d(final v)
        float gca = A.gfin ? A.gfin[2 * r + 1] : 0.0f;  // dL/d(final a)
        // parameter sums: FP32 partials per window, double-single every 4096 steps
        // sums q = 0..4: beta, p, theta0, d, R
#pragma unroll
        for (int q = 0; q < 10; ++q) accs[32 * q] = 0.0f;
        float r_th0 = 0.0f, r_d = 0.0f, r_beta = 0.0f, r_p = 0.0f, r_R = 0.0f;

        for (int wi = (int)A.nwin - 1; wi >= 0; --wi) {
            const long long w = (long long)wi * WIN;
            const int cnt = (int)(A.T - w < WIN ? A.T - w : WIN);
            const bool last_window = wi == (int)A.nwin - 1;
            float x[E], g[E];
            const float *stg = nullptr;  // this window's stage (released at the end of the window)
            if (LOAD == 1) {
                const int st = consumed % NSTAGE;
                if (!mbar_wait_bounded(&bars[st], (consumed / NSTAGE) & 1u)) {
                    report_timeout(A.status);
                    dead = true;
                    break;
                }
                stg = ring + st * STAGE + brow;
#pragma unroll
                for (int q = 0; q < E / 4; ++q) {
                    const int o = 4 * ((ch0 + q) ^ swz);
                    const float4 u = *reinterpret_cast<const float4 *>(stg + o);
                    const float4 v = *reinterpret_cast<const float4 *>(stg + WIN + o);
                    x[4 * q] = u.x; x[4 * q + 1] = u.y; x[4 * q + 2] = u.z; x[4 * q + 3] = u.w;
                    g[4 * q] = v.x; g[4 * q + 1] = v.y; g[4 * q + 2] = v.z; g[4 * q + 3] = v.w;
                }
                if (!GV && !GA) {  // everything this window needs is in registers: refill now
                    __syncwarp();
                    fence_proxy_async_smem();
                    ++consumed;
                    issue();
                }
            } else {
                const long long o = r * A.T + w + t0;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const bool ok = t0 + k < cnt;
                    x[k] = ok ? __ldg(A.I + o + k) : 0.0f;
                    g[k] = ok ? __ldg(A.gS + o + k) : 0.0f;
                }
            }
            if (cnt < WIN) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (t0 + k >= cnt) {
                        x[k] = 0.0f;
                        g[k] = 0.0f;
                    }
            }
            // optional trace-loss gradients at step t0 + k (0 beyond cnt)
            auto trace_grads = [&](float (&gv)[E], float (&gav)[E]) {
#pragma unroll
                for (int k = 0; k < E; ++k) gv[k] = gav[k] = 0.0f;
                if (LOAD == 1) {
#pragma unroll
                    for (int q = 0; q < E / 4; ++q) {
                        const int o = 4 * ((ch0 + q) ^ swz);
                        if (GV) {
                            const float4 u = *reinterpret_cast<const float4 *>(stg + 2 * WIN + o);
                            gv[4 * q] = u.x; gv[4 * q + 1] = u.y; gv[4 * q + 2] = u.z; gv[4 * q + 3] = u.w;
                        }
                        if (GA) {
                            const float4 u = *reinterpret_cast<const float4 *>(stg + (GV ? 3 : 2) * WIN + o);
                            gav[4 * q] = u.x; gav[4 * q + 1] = u.y; gav[4 * q + 2] = u.z; gav[4 * q + 3] = u.w;
                        }
                    }
                } else {
                    const long long o = r * A.T + w + t0;
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        if (GV) gv[k] = __ldg(A.gV + o + k);
                        if (GA) gav[k] = __ldg(A.ga + o + k);
                    }
                }
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (t0 + k >= cnt) gv[k] = gav[k] = 0.0f;
            };

            // ---- state entering the window and this lane's spike bits (loaded one window
            // ahead, so that their latency overlaps the previous window's work)
            const AlifState cs = cs_next;
            const uint32_t wd = wd_next;
            if (wi > 0) {
                cs_next = load_state(wi - 1);
                wd_next = load_word(wi - 1);
            }
            const int rem = cs.rem > 0 ? cs.rem : 0;
            const float vin = rem > 0 ? 0.0f : cs.v;
            const uint32_t sb = (wd >> (t0 & 31)) & FULLM;  // S[t0..t0+E-1]
            const uint32_t up_sb = __shfl_up_sync(FULL, sb, 1);
            const uint32_t prevbit = lane > 0 ? (up_sb >> (E - 1)) & 1u : 0u;  // S[t0-1] (lane 0: in ckpt)

            float s_th0 = 0.0f, s_d = 0.0f, s_beta = 0.0f, s_p = 0.0f, s_R = 0.0f;
            const unsigned spk = __ballot_sync(FULL, sb != 0u);  // lanes holding a spike
            const bool simple = (cnt == WIN) && !last_window && rem == 0 && spk == 0u;
            // The rest of the window, compiled twice.  Lean path (LEAN): a full window without spikes
            // or refractory carry-in, so the mask is 1, there are no resets and cnt = WIN, all known
            // at compile time; V and a decay freely.  General path: ARP mask, segmented scan for V,
            // decayed scan of the shifted spike train for a.
            auto window = [&](auto lean_tag) {
                constexpr bool LEAN = decltype(lean_tag)::value;
                const int cw = LEAN ? WIN : cnt;
                float V[E], a[E], e[E], f[E];
                uint32_t mb = FULLM;  // admitted steps m[t] (bit k)
                const uint32_t rs = LEAN ? 0u : ((sb << 1) | prevbit) & FULLM;  // S[t-1] (reset before step t)
                // ---- V and a
                if constexpr (LEAN) {
                    float q[E];
#pragma unroll
                    for (int j = 0; j < E / 2; ++j) {
                        const float2 u = __fmul2_rn(make_float2(c, c), make_float2(x[2 * j], x[2 * j + 1]));
                        q[2 * j] = u.x;
                        q[2 * j + 1] = u.y;
                    }
                    if (lane == 0) q[0] = fmaf(bf, vin, q[0]);
                    scan_lane<E>(q, V, bf, b4f, Bb);
                    // a = p^t a_w, powers from the lane's anchors (steps 0 and 4)
                    float ak = Pa0 * cs.a;
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        if (k == H) ak = Pa4 * cs.a;
                        a[k] = ak;
                        ak *= pf;
                    }
                } else {
                    // the last spike before the lane (window-relative, -1 = none): the last spike of the
                    // nearest lower lane holding one
                    int lastp;
                    {
                        const unsigned below = spk & ((1u << lane) - 1u);
                        const int top = sb ? t0 + 31 - __clz(sb) : -1;
                        const int tv = __shfl_sync(FULL, top, below ? 31 - __clz(below) : 0);
                        lastp = below ? tv : -1;
                    }
                    {
                        // admitted from the end of the refractory span of the last spike before the lane
                        // (or of the carry-in), up to cnt; then each spike in the lane masks its own span
                        // (spikes fall on admitted steps only, so the spans never overlap the base mask's gaps)
                        const int adm = lastp >= 0 ? lastp + teff : rem;
                        const int h = min(max(cnt - t0, 0), E), l = min(max(adm - t0, 0), E);
                        mb = ((1u << h) - 1u) & ~((1u << l) - 1u);
                        for (uint32_t sp = sb; sp; sp &= sp - 1u) {
                            const int j = __ffs(sp) - 1;
                            const int n = min(teff - 1, E - 1 - j);
                            mb &= ~(((1u << n) - 1u) << (j + 1));
                        }
#pragma unroll
                        for (int k = 0; k < E; ++k)  // from here x holds the admitted input m I
                            if (!((mb >> k) & 1u)) x[k] = 0.0f;
                    }
                    // ---- V: V[t] = beta (1 - S[t-1]) V[t-1] + m c I[t], V entering = vin
                    {
                        // in-lane affine map of the lane's E steps (carry-in 0 for the b part).  The decay
                        // factor of a span of whole lanes is beta^len when no reset falls inside it and 0
                        // otherwise; it is taken from the FP64-derived powers (Bb) instead of being
                        // multiplied up from the rounded beta, whose representation error would grow with
                        // the span.
                        float Ab[E];  // beta (1 - S[t-1])
#pragma unroll
                        for (int k = 0; k < E; ++k) Ab[k] = ((rs >> k) & 1u) ? 0.0f : bf;
                        // the two half lanes' maps (b parts from 0); a half lane's decay is beta^H without
                        // a reset inside it and 0 with one
                        // the window's first input carries beta vin (0 after a refractory carry-in)
                        float cx0 = c * x[0];
                        if (lane == 0) cx0 = fmaf(bf, vin, cx0);
                        float Lb0 = cx0, Lb1 = c * x[H];
#pragma unroll
                        for (int k = 1; k < H; ++k) {
                            Lb0 = fmaf(Ab[k], Lb0, c * x[k]);
                            Lb1 = fmaf(Ab[H + k], Lb1, c * x[H + k]);
                        }
                        const float LA0 = (rs & LOM) ? 0.0f : b4f, LA1 = (rs & HIM) ? 0.0f : b4f;
                        float Lb = fmaf(LA1, Lb0, Lb1);
                        int nr = rs == 0u;  // no reset inside this lane's span
#pragma unroll
                        for (int l = 0; l < 5; ++l) {
                            const int unr = __shfl_up_sync(FULL, nr, 1 << l);
                            const float ub = __shfl_up_sync(FULL, Lb, 1 << l);
                            if (lane >= (1 << l)) {
                                Lb = fmaf(nr ? Bb[l] : 0.0f, ub, Lb);
                                nr &= unr;
                            }
                        }
                        float eb = __shfl_up_sync(FULL, Lb, 1);
                        if (lane == 0) eb = 0.0f;
                        // V[t0-1] carried across lanes (the entering membrane included)
                        float v = eb;
                        const float v3 = fmaf(LA0, v, Lb0);  // V[t0+H-1] from the half-lane decay
#pragma unroll
                        for (int k = 0; k < H - 1; ++k) {
                            v = fmaf(Ab[k], v, k == 0 ? cx0 : c * x[k]);
                            V[k] = v;
                        }
                        V[H - 1] = v3;
                        v = v3;
#pragma unroll
                        for (int k = H; k < E; ++k) {
                            v = fmaf(Ab[k], v, c * x[k]);
                            V[k] = v;
                        }
                        // ---- a: a[t] = p a[t-1] + S[t-1], a[window start] = cs.a
                        float q[E];
#pragma unroll
                        for (int k = 0; k < E; ++k) q[k] = ((rs >> k) & 1u) ? 1.0f : 0.0f;
                        if (lane == 0) q[0] = cs.a;  // a entering the window (S[window start - 1] is inside it)
                        scan_lane<E>(q, a, pf, p4f, Bp);
                    }
                }
                // ---- surrogate and the injections of the reverse recurrences (both paths)
                {
                    float gv[E], gav[E];
                    if (GV || GA) trace_grads(gv, gav);
                    if constexpr (SG == 0) {
                        // fast sigmoid on step pairs with packed f32x2 arithmetic (the reciprocal and
                        // |u| per step); g = 0 beyond cnt, so sgg is too
                        const float2 nd2 = make_float2(-d, -d), nth2 = make_float2(-th0, -th0);
                        float2 sth2 = make_float2(0.0f, 0.0f), sd2 = sth2;
#pragma unroll
                        for (int j = 0; j < E / 2; ++j) {
                            const float2 a2 = make_float2(a[2 * j], a[2 * j + 1]);
                            const float2 u = __ffma2_rn(nd2, a2, __fadd2_rn(make_float2(V[2 * j], V[2 * j + 1]), nth2));
                            const float d0 = fmaf(A.slope, fabsf(u.x), 1.0f), d1 = fmaf(A.slope, fabsf(u.y), 1.0f);
                            const float2 den = __fmul2_rn(make_float2(d0, d1), make_float2(d0, d1));
                            const float2 sgg = __fmul2_rn(make_float2(g[2 * j], g[2 * j + 1]),
                                                          make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y)));
                            sth2 = __fadd2_rn(sth2, sgg);
                            sd2 = __ffma2_rn(a2, sgg, sd2);
                            const float2 e2 = (GV || GA) ? __fadd2_rn(sgg, make_float2(gv[2 * j], gv[2 * j + 1])) : sgg;
                            const float2 f2 = (GV || GA) ? __ffma2_rn(nd2, sgg, make_float2(gav[2 * j], gav[2 * j + 1]))
                                                         : __fmul2_rn(nd2, sgg);
                            e[2 * j] = e2.x;
                            e[2 * j + 1] = e2.y;
                            f[2 * j] = f2.x;
                            f[2 * j + 1] = f2.y;
                        }
                        s_th0 = -(sth2.x + sth2.y);
                        s_d = -(sd2.x + sd2.y);
                    } else {
#pragma unroll
                        for (int k = 0; k < E; ++k) {  // g = 0 beyond cnt, so sgg is too
                            const float u = V[k] - fmaf(d, a[k], th0);
                            const float sgg = surrogate_times<SG>(g[k], u, A.slope);
                            s_th0 -= sgg;
                            s_d = fmaf(-a[k], sgg, s_d);
                            e[k] = (GV || GA) ? sgg + gv[k] : sgg;
                            f[k] = (GV || GA) ? fmaf(-d, sgg, gav[k]) : -d * sgg;
                        }
                    }
                }
                // ---- reverse recurrences: G_V a plain decayed scan on the lean path, segmented
                // (factor beta (1 - S[t]), 0 from step cnt - 1 on) on the general one; G_a decayed
                if constexpr (LEAN) {
                    if (lane == 31) {  // carries from step w + WIN
                        e[E - 1] = fmaf(bf, gcV, e[E - 1]);
                        f[E - 1] = fmaf(pf, gca, f[E - 1]);
                    }
                    rscan_lane<E>(e, bf, b4f, Bb);  // G_V
                } else {
                    {
                        // carries into step cnt - 1 from the next window / the final state; nothing
                        // flows in from beyond the window
                        if (cnt == WIN) {
                            if (lane == 31) {
                                const float Fc = ((sb >> (E - 1)) & 1u) ? 0.0f : (last_window ? 1.0f : bf);
                                e[E - 1] = fmaf(Fc, gcV, e[E - 1]);
                                f[E - 1] = fmaf(pf, gca, f[E - 1]);
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < E; ++k) {
                                const int t = t0 + k;
                                if (t == cnt - 1) {
                                    const float Fc = ((sb >> k) & 1u) ? 0.0f : (last_window ? 1.0f : bf);
                                    e[k] = fmaf(Fc, gcV, e[k]);
                                    f[k] = fmaf(pf, gca, f[k]);
                                }
                            }
                        }
                    }
                    {
                        // reverse affine map of the lane's 8 steps (G_V[t0] = LF G_V[t0+8] + Le); as above,
                        // the decays of spans of whole lanes are exact powers or 0.  Steps whose reverse
                        // factor is 0: a spike, the window's last step and beyond (t0 + k >= cnt - 1), or
                        // every step when beta is 0
                        const int kt = min(max(cnt - 1 - t0, 0), E);
                        unsigned zf = (sb | (FULLM & ~((1u << kt) - 1u))) & FULLM;
                        if (bf == 0.0f) zf = FULLM;
                        float Fr[E];  // the reverse factors
#pragma unroll
                        for (int k = 0; k < E; ++k) Fr[k] = ((zf >> k) & 1u) ? 0.0f : bf;
                        // half lanes: G_V[t0+H] = LF1 G_V[t0+E] + Le1, G_V[t0] = LF0 G_V[t0+H] + Le0
                        float Le0 = 0.0f, Le1 = 0.0f;
#pragma unroll
                        for (int k = H - 1; k >= 0; --k) {
                            Le0 = fmaf(Fr[k], Le0, e[k]);
                            Le1 = fmaf(Fr[H + k], Le1, e[H + k]);
                        }
                        const float LF1 = (zf & HIM) ? 0.0f : b4f;
                        float Le = fmaf((zf & LOM) ? 0.0f : b4f, Le1, Le0);
                        int nr = zf == 0u;
#pragma unroll
                        for (int l = 0; l < 5; ++l) {
                            const int dnr = __shfl_down_sync(FULL, nr, 1 << l);
                            const float de = __shfl_down_sync(FULL, Le, 1 << l);
                            if (lane + (1 << l) < 32) {
                                Le = fmaf(nr ? Bb[l] : 0.0f, de, Le);
                                nr &= dnr;
                            }
                        }
                        float gnext = __shfl_down_sync(FULL, Le, 1);  // G_V[t0+E]
                        if (lane == 31) gnext = 0.0f;
                        float g4 = fmaf(LF1, gnext, Le1);  // G_V[t0+H] from the half-lane decay
#pragma unroll
                        for (int k = E - 1; k > H; --k) {
                            gnext = fmaf(Fr[k], gnext, e[k]);
                            e[k] = gnext;
                        }
                        e[H] = g4;
#pragma unroll
                        for (int k = H - 1; k >= 0; --k) {
                            g4 = fmaf(Fr[k], g4, e[k]);
                            e[k] = g4;
                        }
                    }
                }
                rscan_lane<E>(f, pf, p4f, Bp);  // G_a
                // e = G_V, f = G_a from here

                // ---- dL/dI and the parameter sums (both paths; on the lean path mb is all ones, rs 0)
                {
                    const float Vprev_lane = SAMESTEP ? 0.0f : __shfl_up_sync(FULL, V[E - 1], 1);
                    const float Ga_next_lane = __shfl_down_sync(FULL, f[0], 1);
                    if (A.gI && cw > 0) {
                        float *go = A.gI + r * A.T + w + t0;
                        if (LOAD == 1 && t0 + E <= cw) {
                            const float2 c2 = make_float2(c, c);
#pragma unroll
                            for (int q = 0; q < E / 4; ++q) {
                                const float2 lo = __fmul2_rn(c2, make_float2(e[4 * q], e[4 * q + 1]));
                                const float2 hi = __fmul2_rn(c2, make_float2(e[4 * q + 2], e[4 * q + 3]));
                                float4 o4;
                                o4.x = ((mb >> (4 * q)) & 1u) ? lo.x : 0.0f;
                                o4.y = ((mb >> (4 * q + 1)) & 1u) ? lo.y : 0.0f;
                                o4.z = ((mb >> (4 * q + 2)) & 1u) ? hi.x : 0.0f;
                                o4.w = ((mb >> (4 * q + 3)) & 1u) ? hi.y : 0.0f;
                                reinterpret_cast<float4 *>(go)[q] = o4;
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < E; ++k)
                                if (t0 + k < cw) go[k] = ((mb >> k) & 1u) ? c * e[k] : 0.0f;
                        }
                    }
                    // beyond cnt every term is 0 (x, G_V and G_a vanish there); step pairs, packed.
                    // The beta sum is sum_t (V[t-1] (1 - S[t-1]) - R m I[t]) G_V[t] (the membrane
                    // entering t); with SAMESTEP it is taken as sum_t (V[t] - R m I[t]) G_V[t], which is
                    // beta times it (V[t] - (1 - beta) R m I[t] is beta times the membrane entering t)
                    // and needs no shifted pairs; the 1/beta joins dbeta/dtau below.  For beta < 1/2
                    // that form cancels (V[t] near R m I[t]); those rows' g_tau_mem is recomputed in
                    // the shifted form by the follow-up kernel.
                    float2 sb2 = make_float2(0.0f, 0.0f), sxe2 = sb2, sp2 = sb2;
                    const float2 nR2 = make_float2(-nr.R, -nr.R);
#pragma unroll
                    for (int j = 0; j < E / 2; ++j) {
                        float vp0, vp1;
                        if constexpr (SAMESTEP) {
                            vp0 = V[2 * j];
                            vp1 = V[2 * j + 1];
                        } else {
                            vp0 = j > 0 ? V[2 * j - 1] : (lane > 0 ? Vprev_lane : vin);
                            vp1 = V[2 * j];
                            if ((rs >> (2 * j)) & 1u) vp0 = 0.0f;
                            if ((rs >> (2 * j + 1)) & 1u) vp1 = 0.0f;
                        }
                        const float gan1 = 2 * j + 1 < E - 1 ? f[2 * j + 2] : (lane < 31 ? Ga_next_lane : gca);
                        const float2 x2 = make_float2(x[2 * j], x[2 * j + 1]), e2 = make_float2(e[2 * j], e[2 * j + 1]);
                        sb2 = __ffma2_rn(__ffma2_rn(nR2, x2, make_float2(vp0, vp1)), e2, sb2);
                        sxe2 = __ffma2_rn(x2, e2, sxe2);
                        sp2 = __ffma2_rn(make_float2(a[2 * j], a[2 * j + 1]), make_float2(f[2 * j + 1], gan1), sp2);
                    }
                    s_beta = sb2.x + sb2.y;
                    s_p = sp2.x + sp2.y;
                    const float s_xe = sxe2.x + sxe2.y;
                    if (cw < WIN) {
                        // a partial window: G_a after its last step cnt - 1 is the carry (the loop took
                        // G_a there as 0, its value beyond cnt)
                        const int kl = cw - 1 - t0;
                        if (kl >= 0 && kl < E) {
                            float al = a[0];
#pragma unroll
                            for (int k = 1; k < E; ++k)
                                if (k == kl) al = a[k];
                            s_p = fmaf(al, gca, s_p);
                        }
                    }
                    s_R = nr.one_minus_beta * s_xe;
                }
                gcV = __shfl_sync(FULL, e[0], 0);
                gca = __shfl_sync(FULL, f[0], 0);
            };
            if (simple)
                window(std::true_type{});
            else
                window(std::false_type{});
            if (LOAD == 1 && (GV || GA)) {  // release the stage (trace gradients were read from it)
                __syncwarp();
                fence_proxy_async_smem();
                ++consumed;
                issue();
            }
            r_th0 += s_th0;
            r_d += s_d;
            r_beta += s_beta;
            r_p += s_p;
            r_R += s_R;
            if ((wi & (Geo<E>::FOLD - 1)) == 0) {  // fold 4096 steps of FP32 partials into double-single
                const float rq[5] = {r_beta, r_p, r_th0, r_d, r_R};
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const df u = df_add(df{accs[32 * q], accs[32 * (5 + q)]}, df{rq[q], 0.0f});
                    accs[32 * q] = u.hi;
                    accs[32 * (5 + q)] = u.lo;
                }
                r_th0 = r_d = r_beta = r_p = r_R = 0.0f;
            }
        }
        if (dead) break;
        // deterministic warp reduction of the parameter sums (double-single butterfly)
        df acc[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] = df{accs[32 * q], accs[32 * (5 + q)]};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const df o{__shfl_xor_sync(FULL, acc[q].hi, off), __shfl_xor_sync(FULL, acc[q].lo, off)};
                acc[q] = df_add(acc[q], o);
            }
        }
        if (lane == 0) {
            // per-row partials as (hi, lo) pairs, chained to the time constants
            // the same-step beta sum carries a factor beta: dbeta/dtau / beta = DT / tau^2 (rows with
            // beta < 1/2 are rewritten by the follow-up kernel)
            const float kb = SAMESTEP ? (bf > 0.0f ? nr.dbeta_dtau / bf : 0.0f) : nr.dbeta_dtau;
            const df gtm = df_mul_f(acc[0], kb), gta = df_mul_f(acc[1], nr.dp_dtau);
            float *o = A.part + r * (2 * ALIF_NUM_PARAM_GRADS);
            o[2 * ALIF_G_TAU_MEM] = gtm.hi;
            o[2 * ALIF_G_TAU_MEM + 1] = gtm.lo;
            o[2 * ALIF_G_TAU_ADAPT] = gta.hi;
            o[2 * ALIF_G_TAU_ADAPT + 1] = gta.lo;
            o[2 * ALIF_G_THETA0] = acc[2].hi;
            o[2 * ALIF_G_THETA0 + 1] = acc[2].lo;
            o[2 * ALIF_G_D] = acc[3].hi;
            o[2 * ALIF_G_D + 1] = acc[3].lo;
            o[2 * ALIF_G_R] = acc[4].hi;
            o[2 * ALIF_G_R + 1] = acc[4].lo;
            if (A.ginit) {
                A.ginit[2 * r] = bf * gcV;
                A.ginit[2 * r + 1] = gca;
            }
        }
    }
    if (LOAD == 1) {
        while (consumed < issued) {
            if (!mbar_wait_bounded(&bars[consumed % NSTAGE], (consumed / NSTAGE) & 1u)) {
                report_timeout(A.status);
                break;
            }
            ++consumed;
        }
    }
}

}  // namespace bwd

static int g_sm_count_bwd = 0;
static int g_bwd_window = 0;  // 0: chosen from the row count; 256 or 512: forced

int launch_alif_backward_taumem(long long rows, long long N, long long T, const float *I, const AlifNeuron *nrn,
                                const uint32_t *spikes, const AlifState *ckpt, const AlifState *init,
                                const float *gS, const float *gfin, float slope, float *part, int *status,
                                cudaStream_t stream);

template <int LOAD, bool GV, bool GA, int SG, int E>
static int launch_variant(const CUtensorMap *m, const bwd::Args &A, cudaStream_t stream) {
    using namespace bwd;
    constexpr int smem = smem_bytes<GV, GA, E>();
    static int occ = 0;
    const void *fn = (const void *)bwd_kernel<LOAD, GV, GA, SG, E>;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, WARPS * 32, smem);
        occ = n > 0 ? n : 1;
    }
    const long long need = (A.rows + WARPS - 1) / WARPS;
    const long long cap = (long long)g_sm_count_bwd * occ;
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return 0;
    // the launch's own status (cudaGetLastError could report an earlier, unrelated failure)
    void *args[] = {const_cast<CUtensorMap *>(&m[0]), const_cast<CUtensorMap *>(&m[1]),
                    const_cast<CUtensorMap *>(&m[2]), const_cast<CUtensorMap *>(&m[3]), const_cast<Args *>(&A)};
    return (int)cudaLaunchKernel(fn, dim3(grid), dim3(WARPS * 32), args, smem, stream);
}

template <int SG>
static int dispatch_sel(int sel, bool wide, const CUtensorMap *m, const bwd::Args &A, cudaStream_t stream) {
    if (wide) return launch_variant<1, false, false, SG, 16>(m, A, stream);
    switch (sel) {
        case 0: return launch_variant<0, false, false, SG, 8>(m, A, stream);
        case 1: return launch_variant<0, false, true, SG, 8>(m, A, stream);
        case 2: return launch_variant<0, true, false, SG, 8>(m, A, stream);
        case 3: return launch_variant<0, true, true, SG, 8>(m, A, stream);
        case 4: return launch_variant<1, false, false, SG, 8>(m, A, stream);
        case 5: return launch_variant<1, false, true, SG, 8>(m, A, stream);
        case 6: return launch_variant<1, true, false, SG, 8>(m, A, stream);
        default: return launch_variant<1, true, true, SG, 8>(m, A, stream);
    }
}

int launch_alif_backward(long long B, long long N, long long T, const float *I,
                         const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                         const AlifState *ckpt, const float *gS, const float *gV, const float *ga,
                         const float *gfin, float slope, int surrogate, float *gI, float *ginit,
                         float *part, int *status, cudaStream_t stream) {
    using namespace bwd;
    Args A;
    A.rows = B * N;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS;
    A.I = I;
    A.nrn = nrn;
    A.init = init;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.gS = gS;
    A.gV = gV;
    A.ga = ga;
    A.gfin = gfin;
    A.slope = slope;
    A.gI = gI;
    A.ginit = ginit;
    A.part = part;
    A.status = status;
    if (g_sm_count_bwd == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count_bwd, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count_bwd <= 0) g_sm_count_bwd = 1;
    }
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const long long n16 = A.rows * T / 16;
    bool tma = (T % 16 == 0) && a16(I) && a16(gS) && (!gV || a16(gV)) && (!ga || a16(ga)) &&
               (!gI || a16(gI)) && (n16 + 32 < (1LL << 31));
    // 512-step windows when the rows leave warp slots empty (each row's chain of windows is then the
    // limit, and longer windows halve it), 256-step windows (four CTAs per SM) otherwise; the wide
    // kernel serves the TMA path without trace gradients
    bool wide = g_bwd_window == 512 || (g_bwd_window == 0 && A.rows <= 8LL * g_sm_count_bwd);
    wide = wide && tma && !gV && !ga;
    const unsigned win = wide ? Geo<16>::WIN : Geo<8>::WIN;
    A.nwin = (T + win - 1) / win;
    CUtensorMap m[4];
    memset(m, 0, sizeof m);
    if (tma) {
        tma = make_rows16_map(&m[0], I, n16, win / 16) == 0 && make_rows16_map(&m[1], gS, n16, win / 16) == 0 &&
              (!gV || make_rows16_map(&m[2], gV, n16, win / 16) == 0) &&
              (!ga || make_rows16_map(&m[3], ga, n16, win / 16) == 0);
        if (!tma) {
            memset(m, 0, sizeof m);
            wide = false;
            A.nwin = (T + Geo<8>::WIN - 1) / Geo<8>::WIN;
        }
    }
    const int sel = (tma ? 4 : 0) | (gV ? 2 : 0) | (ga ? 1 : 0);
    switch (surrogate) {
        case 1: return dispatch_sel<1>(sel, wide, m, A, stream);
        case 2: return dispatch_sel<2>(sel, wide, m, A, stream);
        default: break;
    }
    const int rc = dispatch_sel<0>(sel, wide, m, A, stream);
    // the same-step variants (fast sigmoid, no trace gradients, TMA staging) leave g_tau_mem of the
    // rows with beta < 1/2 to the follow-up kernel
    if (rc != 0 || !tma || gV || ga) return rc;
    return launch_alif_backward_taumem(A.rows, N, T, I, nrn, spikes, ckpt, init, gS, gfin, slope, part, status, stream);
}

}  // namespace alif

// Window length of the detached backward (see include/alif.h).
extern "C" int alif_backward_window(int steps) {
    if (steps != 0 && steps != 256 && steps != 512) return ALIF_EINVAL;
    const int prev = alif::g_bwd_window;
    alif::g_bwd_window = steps;
    return prev;
}
