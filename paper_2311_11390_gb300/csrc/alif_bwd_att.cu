// "Attached" surrogate-gradient backward of the blocked ALIF forward (sm_103a).
//
// Attached (Supplementary, "Detaching gradients"): the spike S[t] keeps its
// surrogate gradient where it enters the next step -- the reset factor of
// V[t+1] (Eq 2) and the update a[t+1] = p a[t] + S[t] (Eq 5); the ARP mask
// (Eq 4, an integer step count) still carries none.  With
//     W[t] = beta V[t] + (1 - beta) R m[t+1] I[t+1]   (V[t+1] before its reset factor)
// and sg[t] the surrogate dS/du at u = V[t] - theta[t]:
//     G_S[t] = gS[t] + G_a[t+1] - W[t] G_V[t+1]
//     G_V[t] = gV[t] + sg[t] G_S[t] + beta (1 - S[t]) G_V[t+1]
//     G_a[t] = ga[t] - d sg[t] G_S[t] + p G_a[t+1]
// so (G_V, G_a)[t] = M[t] (G_V, G_a)[t+1] + b[t], a linear recurrence with
//     M[t] = [[beta (1 - S[t]) - sg W, sg], [d sg W, p - d sg]],
//     b[t] = (gV + sg gS, ga - d sg gS)[t].
// One warp owns a row and walks its 512-step windows from the last to the
// first (lane L holds steps 16L .. 16L+15).  Per window it recomputes V and a
// in double-single from the forward's checkpoint and the stored spikes (no
// spike decision is re-taken; the coupled recurrences amplify the surrogate's
// rounding error, so u = V - theta is formed to ~48 bits), composes each
// lane's 16 affine maps, runs a suffix scan of the
// 2 x 2 affine maps across the warp, applies the result to the carry from the
// window after, and accumulates the parameter sums of the detached backward
// with G_S in place of gS.  Inputs are read straight from global memory.
//
// Call boundaries.  The state handed between calls is (v, a) = (V (1 - S),
// p a + S) of the last step, so the last step of a call couples to grad_final
// with W = V[T-1] and reset factor 1 - S.  The remaining part of W, the input
// term (1 - beta) R m I of the next call's first step, is known only to that
// call: it returns -(1 - beta) R m[0] I[0] G_V[0] in grad_init_spike, and the
// call before adds it to dL/dS of its last step as grad_final_spike.  (At
// T_R = 1 the step after a spike is admitted by Eq 4, so m there is 1.)
#include "bwd_scan.cuh"
#include "common.cuh"

namespace alif {
namespace batt {

constexpr int E = BWD_E;
constexpr int WIN = 32 * E;
static_assert(WIN == 2 * ALIF_CKPT_STEPS, "a window spans two checkpoint strides");
constexpr int WARPS = 4;

struct Args {
    long long rows, N, T, nwords, nckpt, nwin;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    const uint32_t *spikes;
    const AlifState *ckpt;
    const float *gS, *gV, *ga, *gfin, *gfin_s;
    float slope;
    float *gI, *ginit, *ginit_s, *part;
};

// x -> A x + c on (G_V, G_a), A = [[a00, a01], [a10, a11]].
struct Aff {
    float a00, a01, a10, a11, c0, c1;
};

// f after g: x -> f(g(x)).
__device__ __forceinline__ Aff compose(const Aff &f, const Aff &g) {
    Aff h;
    h.a00 = fmaf(f.a00, g.a00, f.a01 * g.a10);
    h.a01 = fmaf(f.a00, g.a01, f.a01 * g.a11);
    h.a10 = fmaf(f.a10, g.a00, f.a11 * g.a10);
    h.a11 = fmaf(f.a10, g.a01, f.a11 * g.a11);
    h.c0 = fmaf(f.a00, g.c0, fmaf(f.a01, g.c1, f.c0));
    h.c1 = fmaf(f.a10, g.c0, fmaf(f.a11, g.c1, f.c1));
    return h;
}

// y[t] = A y[t-1] + q(t) over the warp's 512 steps in double-single, with the factor A
// replaced by 0 at the lane steps whose bit is set in `kill`; y before the window is y_in.
// A16 = A^16.  Each lane composes its 16 steps into one affine map, a warp scan of the
// maps gives every lane its entry value, and the lane replays its steps from it.
template <class QF>
__device__ __forceinline__ void df_affine_scan(df Af, df A16, uint32_t kill, QF q, df y_in, int lane,
                                               float (&yh)[E], float (&yl)[E]) {
    df Lb{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < E; ++k) Lb = ((kill >> k) & 1u) ? q(k) : df_add(df_mul(Af, Lb), q(k));
    df LA = (kill & 0xffffu) ? df{0.0f, 0.0f} : A16;
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const df uA{__shfl_up_sync(FULL, LA.hi, 1 << l), __shfl_up_sync(FULL, LA.lo, 1 << l)};
        const df ub{__shfl_up_sync(FULL, Lb.hi, 1 << l), __shfl_up_sync(FULL, Lb.lo, 1 << l)};
        if (lane >= (1 << l)) {
            Lb = df_add(df_mul(LA, ub), Lb);
            LA = df_mul(LA, uA);
        }
    }
    const df pA{__shfl_up_sync(FULL, LA.hi, 1), __shfl_up_sync(FULL, LA.lo, 1)};
    const df pb{__shfl_up_sync(FULL, Lb.hi, 1), __shfl_up_sync(FULL, Lb.lo, 1)};
    df y = lane == 0 ? y_in : df_add(df_mul(pA, y_in), pb);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        y = ((kill >> k) & 1u) ? q(k) : df_add(df_mul(Af, y), q(k));
        yh[k] = y.hi;
        yl[k] = y.lo;
    }
}

template <int SG>
__global__ void __launch_bounds__(WARPS * 32) bwd_att_kernel(const Args A) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long nw = (long long)gridDim.x * WARPS;
    const int t0 = E * lane;
    for (long long r = gw; r < A.rows; r += nw) {
        const AlifNeuron nr = A.nrn[r % A.N];
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        const float bf = beta.hi, pf = p.hi, c = nr.c_hi, d = nr.d, th0 = nr.theta0;
        const int teff = nr.teff;
        const bool tr1 = nr.tr == 1;
        const df b16 = df_pow(beta, E), p16 = df_pow(p, E), cdf{nr.c_hi, nr.c_lo};
        const uint32_t *bits = A.spikes + r * A.nwords;
        float gcV = A.gfin ? A.gfin[2 * r] : 0.0f;      // (G_V, G_a) just after the window
        float gca = A.gfin ? A.gfin[2 * r + 1] : 0.0f;
        float Vn0 = 0.0f, xn0 = 0.0f;  // V and the raw input at the first step of the window after
        bool m0 = false;               // that step admitted (Eq 4)
        df acc_th0{0.0f, 0.0f}, acc_d{0.0f, 0.0f}, acc_beta{0.0f, 0.0f}, acc_p{0.0f, 0.0f}, acc_R{0.0f, 0.0f};
        float r_th0 = 0.0f, r_d = 0.0f, r_beta = 0.0f, r_p = 0.0f, r_R = 0.0f;

        for (int wi = (int)A.nwin - 1; wi >= 0; --wi) {
            const long long w = (long long)wi * WIN;
            const int cnt = (int)(A.T - w < WIN ? A.T - w : WIN);
            const bool last_window = wi == (int)A.nwin - 1;
            const long long o = r * A.T + w + t0;
            float x[E], g[E];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const bool ok = t0 + k < cnt;
                x[k] = ok ? __ldg(A.I + o + k) : 0.0f;
                g[k] = ok ? __ldg(A.gS + o + k) : 0.0f;
            }
            if (last_window && A.gfin_s) {  // dL/dS of the last step from the next call's input term
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (t0 + k == cnt - 1) g[k] += A.gfin_s[r];
            }
            AlifState cs{0.0f, 0.0f, 0};
            if (A.ckpt)
                cs = A.ckpt[r * A.nckpt + 2LL * wi];
            else if (A.init)
                cs = A.init[r];
            const int rem = cs.rem > 0 ? cs.rem : 0;
            const float vin = rem > 0 ? 0.0f : cs.v;
            const long long widx = (long long)wi * (WIN / 32) + (lane >> 1);
            const uint32_t wd = widx < A.nwords ? __ldg(bits + widx) : 0u;
            uint32_t sb = (wd >> (16 * (lane & 1))) & 0xffffu;  // S[t0 .. t0+15]
            {
                const int nv = cnt - t0;
                if (nv < E) sb &= nv > 0 ? (1u << nv) - 1u : 0u;
            }
            const uint32_t up_sb = __shfl_up_sync(FULL, sb, 1);
            const uint32_t prevbit = lane > 0 ? (up_sb >> 15) & 1u : 0u;  // S[t0-1] (lane 0: in ckpt)
            const uint32_t rs = ((sb << 1) | prevbit) & 0xffffu;            // S[t-1]

            // W[t] is assembled in Wt: first the admitted input of the step after a spike
            // (T_R = 1 only; raw, before the mask below removes it), later beta V[t] or V[t+1]
            float Wt[E];
            const float x0raw = __shfl_sync(FULL, x[0], 0);
            {
                const float xup = __shfl_down_sync(FULL, x[0], 1);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const float xnext = k < E - 1 ? x[k + 1] : (lane < 31 ? xup : xn0);
                    Wt[k] = (tr1 && ((sb >> k) & 1u)) ? c * xnext : 0.0f;
                }
            }
            // ---- admitted steps m[t] (bit k) and the masked input
            int lastp;
            {
                int incl = sb ? t0 + 31 - __clz(sb) : -1;
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const int upv = __shfl_up_sync(FULL, incl, 1 << l);
                    if (lane >= (1 << l)) incl = max(incl, upv);
                }
                lastp = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) lastp = -1;
            }
            uint32_t mb = 0;
            {
                int lp = lastp;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int t = t0 + k;
                    if ((lp >= 0 ? (t >= lp + teff) : (t >= rem)) && (t < cnt)) mb |= 1u << k;
                    if ((sb >> k) & 1u) lp = t;
                }
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (!((mb >> k) & 1u)) x[k] = 0.0f;
            }
            // ---- V[t] = beta (1 - S[t-1]) V[t-1] + m c I[t] from V entering = vin, and
            // a[t] = p a[t-1] + S[t-1] from a at the window start = cs.a, both in double-single:
            // the attached recurrences feed the surrogate's rounding error back through G_V and
            // G_a, so u = V - theta is formed from ~48-bit V and a
            float V[E], a[E], uu[E];
            {
                float ah[E], al[E], vh[E], vl[E];
                // cs.a is a at the window's first step itself: lane 0 starts its chain there
                df_affine_scan(
                    p, p16, lane == 0 ? 1u : 0u,
                    [&](int k) {
                        return (lane == 0 && k == 0) ? df{cs.a, 0.0f}
                                                     : df{((rs >> k) & 1u) ? 1.0f : 0.0f, 0.0f};
                    },
                    df{0.0f, 0.0f}, lane, ah, al);
                df_affine_scan(beta, b16, rs, [&](int k) { return df_mul_f(cdf, x[k]); }, df{vin, 0.0f}, lane,
                               vh, vl);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const df th = df_add(df{th0, 0.0f}, df_mul_f(df{ah[k], al[k]}, d));
                    const df u = df_add(df{vh[k], vl[k]}, df_neg(th));
                    uu[k] = u.hi + u.lo;
                    V[k] = vh[k];
                    a[k] = ah[k];
                }
            }
            // ---- surrogate, W, injections
            float sg[E], bV[E], bA[E];
            {
                const float Vup = __shfl_down_sync(FULL, V[0], 1);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int t = t0 + k;
                    sg[k] = t < cnt ? surrogate_times<SG>(1.0f, uu[k], A.slope) : 0.0f;
                    const float Vnext = k < E - 1 ? V[k + 1] : (lane < 31 ? Vup : Vn0);
                    Wt[k] = ((sb >> k) & 1u) ? fmaf(bf, V[k], Wt[k]) : Vnext;
                    if (last_window && t == cnt - 1) Wt[k] = V[k];  // final state v = V (1 - S)
                    const float gv = (A.gV && t < cnt) ? __ldg(A.gV + o + k) : 0.0f;
                    const float gav = (A.ga && t < cnt) ? __ldg(A.ga + o + k) : 0.0f;
                    bV[k] = fmaf(sg[k], g[k], gv);
                    bA[k] = fmaf(-d * sg[k], g[k], gav);
                }
            }
            // M[t] of step k (identity beyond cnt, so that the carry reaches step cnt - 1)
            auto step_map = [&](int k) {
                const int t = t0 + k;
                Aff m;
                if (t >= cnt) {
                    m = Aff{1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
                } else {
                    const float F = ((sb >> k) & 1u) ? 0.0f : ((last_window && t == cnt - 1) ? 1.0f : bf);
                    const float s = sg[k], sW = s * Wt[k];
                    m = Aff{F - sW, s, d * sW, fmaf(-d, s, pf), bV[k], bA[k]};
                }
                return m;
            };
            // ---- lane maps (step t0+16 -> step t0), warp suffix scan, apply to the carry
            Aff L{1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = E - 1; k >= 0; --k) L = compose(step_map(k), L);
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                Aff U;
                U.a00 = __shfl_down_sync(FULL, L.a00, 1 << l);
                U.a01 = __shfl_down_sync(FULL, L.a01, 1 << l);
                U.a10 = __shfl_down_sync(FULL, L.a10, 1 << l);
                U.a11 = __shfl_down_sync(FULL, L.a11, 1 << l);
                U.c0 = __shfl_down_sync(FULL, L.c0, 1 << l);
                U.c1 = __shfl_down_sync(FULL, L.c1, 1 << l);
                if (lane + (1 << l) < 32) L = compose(L, U);
            }
            const float at0V = fmaf(L.a00, gcV, fmaf(L.a01, gca, L.c0));  // G_V[t0]
            const float at0A = fmaf(L.a10, gcV, fmaf(L.a11, gca, L.c1));  // G_a[t0]
            float nV = __shfl_down_sync(FULL, at0V, 1), nA = __shfl_down_sync(FULL, at0A, 1);
            if (lane == 31) {
                nV = gcV;
                nA = gca;
            }
            // ---- in-lane reverse pass: bV/bA become G_V/G_a; theta0, d and p sums
            float s_th0 = 0.0f, s_d = 0.0f, s_p = 0.0f;
#pragma unroll
            for (int k = E - 1; k >= 0; --k) {
                const Aff m = step_map(k);
                const float GV = fmaf(m.a00, nV, fmaf(m.a01, nA, m.c0));
                const float GA = fmaf(m.a10, nV, fmaf(m.a11, nA, m.c1));
                if (t0 + k < cnt) {
                    const float sgs = sg[k] * (g[k] + nA - Wt[k] * nV);  // sg G_S
                    s_th0 -= sgs;
                    s_d = fmaf(-a[k], sgs, s_d);
                    s_p = fmaf(a[k], nA, s_p);  // a[t] G_a[t+1]
                }
                bV[k] = GV;
                bA[k] = GA;
                nV = GV;
                nA = GA;
            }
            // ---- dL/dI, beta and R sums
            float s_beta = 0.0f, s_xe = 0.0f;
            {
                const float Vprev_lane = __shfl_up_sync(FULL, V[E - 1], 1);
                float *go = A.gI ? A.gI + o : nullptr;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    if (t0 + k < cnt) {
                        float vprev = k > 0 ? V[k - 1] : (lane > 0 ? Vprev_lane : vin);
                        if ((rs >> k) & 1u) vprev = 0.0f;
                        s_beta = fmaf(fmaf(-nr.R, x[k], vprev), bV[k], s_beta);
                        s_xe = fmaf(x[k], bV[k], s_xe);
                        if (go) go[k] = ((mb >> k) & 1u) ? c * bV[k] : 0.0f;
                    }
                }
            }
            gcV = __shfl_sync(FULL, bV[0], 0);
            gca = __shfl_sync(FULL, bA[0], 0);
            Vn0 = __shfl_sync(FULL, V[0], 0);
            xn0 = x0raw;
            m0 = __shfl_sync(FULL, mb & 1u, 0) != 0u;
            r_th0 += s_th0;
            r_d += s_d;
            r_beta += s_beta;
            r_p += s_p;
            r_R += nr.one_minus_beta * s_xe;
            if ((wi & 7) == 0) {  // fold 8 windows of FP32 partials into double-single
                acc_th0 = df_add(acc_th0, df{r_th0, 0.0f});
                acc_d = df_add(acc_d, df{r_d, 0.0f});
                acc_beta = df_add(acc_beta, df{r_beta, 0.0f});
                acc_p = df_add(acc_p, df{r_p, 0.0f});
                acc_R = df_add(acc_R, df{r_R, 0.0f});
                r_th0 = r_d = r_beta = r_p = r_R = 0.0f;
            }
        }
        // deterministic warp reduction of the parameter sums (double-single butterfly)
        df acc[5] = {acc_beta, acc_p, acc_th0, acc_d, acc_R};
#pragma unroll
        for (int q = 0; q < 5; ++q) {
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const df o2{__shfl_xor_sync(FULL, acc[q].hi, off), __shfl_xor_sync(FULL, acc[q].lo, off)};
                acc[q] = df_add(acc[q], o2);
            }
        }
        if (lane == 0) {
            const df gtm = df_mul_f(acc[0], nr.dbeta_dtau), gta = df_mul_f(acc[1], nr.dp_dtau);
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
            if (A.ginit_s) A.ginit_s[r] = (tr1 || m0) ? -c * xn0 * gcV : 0.0f;
        }
    }
}

}  // namespace batt

template <int SG>
static int launch_att(const batt::Args &A, cudaStream_t stream) {
    using namespace batt;
    static int cap = 0;
    if (cap == 0) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bwd_att_kernel<SG>, WARPS * 32, 0);
        cap = (sms > 0 ? sms : 1) * (occ > 0 ? occ : 1);
    }
    const long long need = (A.rows + WARPS - 1) / WARPS;
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return 0;
    bwd_att_kernel<SG><<<grid, WARPS * 32, 0, stream>>>(A);
    return (int)cudaGetLastError();
}

int launch_alif_backward_attached(long long B, long long N, long long T, const float *I, const AlifNeuron *nrn,
                                  const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                                  const float *gS, const float *gV, const float *ga, const float *gfin,
                                  const float *gfin_s, float slope, int surrogate, float *gI, float *ginit,
                                  float *ginit_s, float *part, cudaStream_t stream) {
    batt::Args A;
    A.rows = B * N;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS;
    A.nwin = (T + batt::WIN - 1) / batt::WIN;
    A.I = I;
    A.nrn = nrn;
    A.init = init;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.gS = gS;
    A.gV = gV;
    A.ga = ga;
    A.gfin = gfin;
    A.gfin_s = gfin_s;
    A.slope = slope;
    A.gI = gI;
    A.ginit = ginit;
    A.ginit_s = ginit_s;
    A.part = part;
    switch (surrogate) {
        case 1: return launch_att<1>(A, stream);
        case 2: return launch_att<2>(A, stream);
        default: return launch_att<0>(A, stream);
    }
}

}  // namespace alif
