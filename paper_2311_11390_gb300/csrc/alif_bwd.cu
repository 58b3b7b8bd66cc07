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
// One warp owns a row and walks its 256-step windows from the last to the
// first (lane L holds steps 8L..8L+7).  For each window it recomputes V and a
// from the checkpoint saved by the forward (state entering the window) and the
// stored spike bits -- no spike decision is re-taken -- then runs both reverse
// recurrences as warp scans and accumulates the parameter gradients.
// Inputs are staged by 1-D bulk copies into a per-warp ring, newest window
// first.  Per-row partial parameter sums go to the workspace; a second kernel
// sums them over the batch in a fixed order (deterministic).
#include "common.cuh"

namespace alif {
namespace bwd {

constexpr int E = 8;
constexpr int WIN = 32 * E;
constexpr int NSTAGE = 3;
constexpr int WARPS = 4;
constexpr int MAXARR = 4;  // I, gS, gV, ga
static_assert(WIN == ALIF_CKPT_STEPS, "window must equal the checkpoint stride");

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
    int narr;  // staged arrays per window: 2 + (gV != 0) + (ga != 0)
};

// Inclusive decayed scan with uniform decay (see the forward kernel).
__device__ __forceinline__ void decay_scan(float (&v)[E], float dec, const float (&Bl)[5],
                                           const float (&dk1)[E], int lane) {
#pragma unroll
    for (int k = 1; k < E; ++k) v[k] = fmaf(dec, v[k - 1], v[k]);
    float tot = v[E - 1];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const float up = __shfl_up_sync(FULL, tot, 1 << l);
        if (lane >= (1 << l)) tot = fmaf(Bl[l], up, tot);
    }
    float P = __shfl_up_sync(FULL, tot, 1);
    if (lane == 0) P = 0.0f;
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = fmaf(dk1[k], P, v[k]);
}

// Reverse decayed scan with uniform decay: v[t] <- sum_{j>=t} dec^{j-t} v[j].
__device__ __forceinline__ void decay_scan_rev(float (&v)[E], float dec, const float (&Bl)[5],
                                               const float (&dk1)[E], int lane) {
#pragma unroll
    for (int k = E - 2; k >= 0; --k) v[k] = fmaf(dec, v[k + 1], v[k]);
    float tot = v[0];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const float dn = __shfl_down_sync(FULL, tot, 1 << l);
        if (lane + (1 << l) < 32) tot = fmaf(Bl[l], dn, tot);
    }
    float P = __shfl_down_sync(FULL, tot, 1);
    if (lane == 31) P = 0.0f;
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = fmaf(dk1[E - 1 - k], P, v[k]);
}

template <bool BULK>
__global__ void __launch_bounds__(WARPS * 32, 3) bwd_kernel(const Args A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stage_floats = A.narr * WIN;
    float *ring = reinterpret_cast<float *>(smem) + (size_t)warp * NSTAGE * MAXARR * WIN;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)WARPS * NSTAGE * MAXARR * WIN * 4) +
                     warp * NSTAGE;
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long nw = (long long)gridDim.x * WARPS;
    if (gw >= A.rows) return;

    const float *src[MAXARR] = {A.I, A.gS, A.gV ? A.gV : A.ga, A.ga};
    // ---- producer: windows newest first, rows in order
    long long p_row = gw, p_wi = A.nwin - 1;
    unsigned issued = 0, consumed = 0;
    uint64_t pol = 0;
    if (BULK) {
        if (lane == 0) {
            for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
        pol = policy_evict_first();
    }
    auto issue = [&]() {
        while (p_row < A.rows && issued - consumed < (unsigned)NSTAGE) {
            const int st = issued % NSTAGE;
            const long long w0 = p_wi * WIN;
            const long long left = A.T - w0;
            const uint32_t bytes = (uint32_t)((left < WIN ? left : WIN) * 4);
            if (lane == 0) {
                mbar_arrive_expect_tx(&bars[st], bytes * (uint32_t)A.narr);
                for (int q = 0; q < A.narr; ++q)
                    bulk_g2s_stream(ring + st * stage_floats + q * WIN, src[q] + p_row * A.T + w0, bytes,
                                    &bars[st], pol);
            }
            ++issued;
            if (--p_wi < 0) {
                p_wi = A.nwin - 1;
                p_row += nw;
            }
        }
    };
    if (BULK) issue();

    const int t0 = 8 * lane;
    bool dead = false;
    for (long long r = gw; r < A.rows && !dead; r += nw) {
        const AlifNeuron nr = A.nrn[r % A.N];
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        float Pw[E], pk1[E], Blp[5], bkb[E], Blb[5], B0b;
        {
            df q = df_pow(p, t0), u = p, ub = beta;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                Pw[k] = q.hi;    // p^t
                pk1[k] = u.hi;   // p^{k+1}
                bkb[k] = ub.hi;  // beta^{k+1}
                q = df_mul(q, p);
                u = df_mul(u, p);
                ub = df_mul(ub, beta);
            }
            B0b = df_pow(beta, t0).hi;  // beta^{8L}
            df p8 = df_pow(p, 8), b8 = df_pow(beta, 8);
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                Blp[l] = p8.hi;
                Blb[l] = b8.hi;
                p8 = df_mul(p8, p8);
                b8 = df_mul(b8, b8);
            }
        }
        const float bf = beta.hi, pf = p.hi, c = nr.c_hi, d = nr.d, th0 = nr.theta0;
        const int teff = nr.teff;
        const uint32_t *bits = A.spikes + r * A.nwords;

        float gcV = A.gfin ? A.gfin[2 * r] : 0.0f;      // dL/d(final v)
        float gca = A.gfin ? A.gfin[2 * r + 1] : 0.0f;  // dL/d(final a)
        // parameter sums: FP32 partials per window, double-single across windows
        df acc_th0{0.0f, 0.0f}, acc_d{0.0f, 0.0f}, acc_beta{0.0f, 0.0f}, acc_p{0.0f, 0.0f}, acc_R{0.0f, 0.0f};
        float r_th0 = 0.0f, r_d = 0.0f, r_beta = 0.0f, r_p = 0.0f, r_R = 0.0f;  // last <= 16 windows
        float GV0 = 0.0f, Ga0 = 0.0f;

        for (long long wi = A.nwin - 1; wi >= 0; --wi) {
            const long long w = wi * WIN;
            const int cnt = (int)(A.T - w < WIN ? A.T - w : WIN);
            const bool last_window = (wi == A.nwin - 1);
            float x[E], g[E], gv[E], gav[E];
            if (BULK) {
                const int st = consumed % NSTAGE;
                if (!mbar_wait_bounded(&bars[st], (consumed / NSTAGE) & 1u)) {
                    report_timeout(A.status);
                    dead = true;
                    break;
                }
                const float *base = ring + st * stage_floats + t0;
#pragma unroll
                for (int k = 0; k < E; k += 4) {
                    const float4 u = *reinterpret_cast<const float4 *>(base + k);
                    const float4 v = *reinterpret_cast<const float4 *>(base + WIN + k);
                    x[k] = u.x; x[k + 1] = u.y; x[k + 2] = u.z; x[k + 3] = u.w;
                    g[k] = v.x; g[k + 1] = v.y; g[k + 2] = v.z; g[k + 3] = v.w;
                }
                int q = 2;
                if (A.gV) {
#pragma unroll
                    for (int k = 0; k < E; k += 4) {
                        const float4 u = *reinterpret_cast<const float4 *>(base + q * WIN + k);
                        gv[k] = u.x; gv[k + 1] = u.y; gv[k + 2] = u.z; gv[k + 3] = u.w;
                    }
                    ++q;
                }
                if (A.ga) {
#pragma unroll
                    for (int k = 0; k < E; k += 4) {
                        const float4 u = *reinterpret_cast<const float4 *>(base + q * WIN + k);
                        gav[k] = u.x; gav[k + 1] = u.y; gav[k + 2] = u.z; gav[k + 3] = u.w;
                    }
                }
                __syncwarp();
                fence_proxy_async_smem();
                ++consumed;
                issue();
            } else {
                const long long o = r * A.T + w + t0;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const bool ok = t0 + k < cnt;
                    x[k] = ok ? __ldg(A.I + o + k) : 0.0f;
                    g[k] = ok ? __ldg(A.gS + o + k) : 0.0f;
                    gv[k] = (ok && A.gV) ? __ldg(A.gV + o + k) : 0.0f;
                    gav[k] = (ok && A.ga) ? __ldg(A.ga + o + k) : 0.0f;
                }
            }
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if (t0 + k >= cnt) {
                    x[k] = 0.0f;
                    g[k] = 0.0f;
                    gv[k] = 0.0f;
                    gav[k] = 0.0f;
                }
                if (!A.gV) gv[k] = 0.0f;
                if (!A.ga) gav[k] = 0.0f;
            }

            // ---- state entering the window and this lane's spike bits
            AlifState cs;
            if (A.ckpt) {
                cs = A.ckpt[r * A.nckpt + wi];
            } else {
                cs = AlifState{0.0f, 0.0f, 0};
                if (A.init) cs = A.init[r];
            }
            const int rem = cs.rem > 0 ? cs.rem : 0;
            const float vin = rem > 0 ? 0.0f : cs.v;
            const long long widx = wi * E + (lane >> 2);
            const uint32_t wd = widx < A.nwords ? __ldg(bits + widx) : 0u;
            const uint32_t sb = (wd >> (t0 & 31)) & 0xffu;  // S[t0..t0+7]
            const uint32_t up_sb = __shfl_up_sync(FULL, sb, 1);
            const uint32_t prevbit = lane > 0 ? (up_sb >> 7) & 1u : 0u;  // S[t0-1] (lane 0: in ckpt)

            float s_th0 = 0.0f, s_d = 0.0f, s_beta = 0.0f, s_p = 0.0f, s_R = 0.0f;
            const bool simple = (cnt == WIN) && !last_window && rem == 0 && __ballot_sync(FULL, sb != 0u) == 0u;
            if (simple) {
                // No spike in the window and no refractory carry-in: the mask is 1, V and a
                // decay freely, G_V and G_a are plain decayed reverse scans.
                float V[E], a[E], e[E], f[E], sgg[E];
                {
#pragma unroll
                    for (int k = 0; k < E; ++k) V[k] = c * x[k];
                    decay_scan(V, bf, Blb, bkb, lane);
                    const float BV = B0b * vin;
#pragma unroll
                    for (int k = 0; k < E; ++k) {
                        V[k] = fmaf(bkb[k], BV, V[k]);
                        a[k] = Pw[k] * cs.a;
                    }
                }
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const float u = V[k] - fmaf(d, a[k], th0);
                    const float den = fmaf(A.slope, fabsf(u), 1.0f);
                    sgg[k] = __fdividef(g[k], den * den);
                    e[k] = sgg[k] + gv[k];
                    f[k] = fmaf(-d, sgg[k], gav[k]);
                }
                if (lane == 31) {  // carries from step w + 256
                    e[E - 1] = fmaf(bf, gcV, e[E - 1]);
                    f[E - 1] = fmaf(pf, gca, f[E - 1]);
                }
                decay_scan_rev(e, bf, Blb, bkb, lane);  // G_V
                decay_scan_rev(f, pf, Blp, pk1, lane);  // G_a
                if (A.gI) {
                    float *go = A.gI + r * A.T + w + t0;
                    if (BULK) {
                        reinterpret_cast<float4 *>(go)[0] = make_float4(c * e[0], c * e[1], c * e[2], c * e[3]);
                        reinterpret_cast<float4 *>(go)[1] = make_float4(c * e[4], c * e[5], c * e[6], c * e[7]);
                    } else {
#pragma unroll
                        for (int k = 0; k < E; ++k) go[k] = c * e[k];
                    }
                }
                const float Vprev_lane = __shfl_up_sync(FULL, V[E - 1], 1);
                const float Ga_next_lane = __shfl_down_sync(FULL, f[0], 1);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const float vprev = k > 0 ? V[k - 1] : (lane > 0 ? Vprev_lane : vin);
                    s_th0 -= sgg[k];
                    s_d = fmaf(-a[k], sgg[k], s_d);
                    s_beta = fmaf(fmaf(-nr.R, x[k], vprev), e[k], s_beta);
                    s_R = fmaf(nr.one_minus_beta * x[k], e[k], s_R);
                    const float gan = k < E - 1 ? f[k + 1] : (lane < 31 ? Ga_next_lane : gca);
                    s_p = fmaf(a[k], gan, s_p);
                }
                gcV = __shfl_sync(FULL, e[0], 0);
                gca = __shfl_sync(FULL, f[0], 0);
            } else {
            // last spike strictly before each element (window-relative, -1 = none)
            int lastp;
            {
                int mine = sb ? t0 + 31 - __clz(sb) : -1;
                int incl = mine;
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const int up = __shfl_up_sync(FULL, incl, 1 << l);
                    if (lane >= (1 << l)) incl = max(incl, up);
                }
                lastp = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) lastp = -1;
            }
            float m[E];
            {
                int lp = lastp;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int t = t0 + k;
                    m[k] = (lp >= 0 ? (t >= lp + teff) : (t >= rem)) && (t < cnt) ? 1.0f : 0.0f;
                    if ((sb >> k) & 1u) lp = t;
                }
            }

            // ---- V: V[t] = beta (1 - S[t-1]) V[t-1] + m c I[t], V[-1] -> vin
            float V[E];
            {
                float Ac[E], bc[E];
                float Ak = bf, bk = m[0] * c * x[0];
                // element 0's factor uses S[t0-1] from the previous lane
                if (prevbit) Ak = 0.0f;
                Ac[0] = Ak;
                bc[0] = bk;
#pragma unroll
                for (int k = 1; k < E; ++k) {
                    const float Af = ((sb >> (k - 1)) & 1u) ? 0.0f : bf;
                    Ac[k] = Af * Ac[k - 1];
                    bc[k] = fmaf(Af, bc[k - 1], m[k] * c * x[k]);
                }
                float LA = Ac[E - 1], Lb = bc[E - 1];
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const float uA = __shfl_up_sync(FULL, LA, 1 << l);
                    const float ub = __shfl_up_sync(FULL, Lb, 1 << l);
                    if (lane >= (1 << l)) {
                        Lb = fmaf(LA, ub, Lb);
                        LA = LA * uA;
                    }
                }
                float eA = __shfl_up_sync(FULL, LA, 1), eb = __shfl_up_sync(FULL, Lb, 1);
                if (lane == 0) {
                    eA = 1.0f;
                    eb = 0.0f;
                }
                const float Venter = fmaf(eA, vin, eb);  // V[t0-1] (reset applied via Ac)
#pragma unroll
                for (int k = 0; k < E; ++k) V[k] = fmaf(Ac[k], Venter, bc[k]);
            }

            // ---- a: a[t] = p a[t-1] + S[t-1], a[0] = a_w
            float a[E];
            {
                const unsigned y = ((sb << 1) | prevbit) & 0xffu;  // S[t-1]
#pragma unroll
                for (int k = 0; k < E; ++k) a[k] = ((y >> k) & 1u) ? 1.0f : 0.0f;
                decay_scan(a, pf, Blp, pk1, lane);
#pragma unroll
                for (int k = 0; k < E; ++k) a[k] = fmaf(Pw[k], cs.a, a[k]);
            }

            // ---- surrogate, injections, reverse recurrences
            float e[E], f[E], F[E], sgg[E];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int t = t0 + k;
                const float u = V[k] - fmaf(d, a[k], th0);
                const float den = fmaf(A.slope, fabsf(u), 1.0f);
                const float sg = __fdividef(1.0f, den * den);
                sgg[k] = sg * g[k];
                e[k] = sgg[k] + gv[k];
                f[k] = fmaf(-d, sgg[k], gav[k]);
                const bool S = (sb >> k) & 1u;
                F[k] = S ? 0.0f : ((last_window && t == cnt - 1) ? 1.0f : bf);
                if (t >= cnt) F[k] = 1.0f;
                if (t == cnt - 1) {
                    e[k] = fmaf(F[k], gcV, e[k]);  // carry from the next window / final state
                    f[k] = fmaf(pf, gca, f[k]);
                }
            }
            float GV[E];
            {
                float Fc[E], ec[E];
                Fc[E - 1] = F[E - 1];
                ec[E - 1] = e[E - 1];
#pragma unroll
                for (int k = E - 2; k >= 0; --k) {
                    Fc[k] = F[k] * Fc[k + 1];
                    ec[k] = fmaf(F[k], ec[k + 1], e[k]);
                }
                float LF = Fc[0], Le = ec[0];
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const float dF = __shfl_down_sync(FULL, LF, 1 << l);
                    const float de = __shfl_down_sync(FULL, Le, 1 << l);
                    if (lane + (1 << l) < 32) {
                        Le = fmaf(LF, de, Le);
                        LF = LF * dF;
                    }
                }
                float right = __shfl_down_sync(FULL, Le, 1);  // G_V[t0+8]
                if (lane == 31) right = 0.0f;
#pragma unroll
                for (int k = 0; k < E; ++k) GV[k] = fmaf(Fc[k], right, ec[k]);
            }
            float Ga[E];
#pragma unroll
            for (int k = 0; k < E; ++k) Ga[k] = f[k];
            {
                float pk1r[E];
#pragma unroll
                for (int k = 0; k < E; ++k) pk1r[k] = pk1[k];
                decay_scan_rev(Ga, pf, Blp, pk1r, lane);
            }

            // ---- outputs and parameter sums
            const float Vprev_lane = __shfl_up_sync(FULL, V[E - 1], 1);
            const float Ga_next_lane = __shfl_down_sync(FULL, Ga[0], 1);
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int t = t0 + k;
                if (t < cnt) {
                    const float gi = c * m[k] * GV[k];
                    if (A.gI) A.gI[r * A.T + w + t] = gi;
                    const bool Sp = k > 0 ? ((sb >> (k - 1)) & 1u) : prevbit;
                    float vprev = k > 0 ? V[k - 1] : (lane > 0 ? Vprev_lane : vin);
                    if (Sp) vprev = 0.0f;
                    const float Iin = m[k] * x[k];
                    s_th0 -= sgg[k];
                    s_d = fmaf(-a[k], sgg[k], s_d);
                    s_beta = fmaf(fmaf(-nr.R, Iin, vprev), GV[k], s_beta);
                    s_R = fmaf(nr.one_minus_beta * Iin, GV[k], s_R);
                    const float gan = (t == cnt - 1) ? gca : (k < E - 1 ? Ga[k + 1] : Ga_next_lane);
                    s_p = fmaf(a[k], gan, s_p);
                }
            }
            // carries into the previous window
            gcV = __shfl_sync(FULL, GV[0], 0);
            gca = __shfl_sync(FULL, Ga[0], 0);
            }
            GV0 = gcV;
            Ga0 = gca;
            r_th0 += s_th0;
            r_d += s_d;
            r_beta += s_beta;
            r_p += s_p;
            r_R += s_R;
            if ((wi & 15) == 0) {  // fold 16 windows of FP32 partials into double-single
                acc_th0 = df_add(acc_th0, df{r_th0, 0.0f});
                acc_d = df_add(acc_d, df{r_d, 0.0f});
                acc_beta = df_add(acc_beta, df{r_beta, 0.0f});
                acc_p = df_add(acc_p, df{r_p, 0.0f});
                acc_R = df_add(acc_R, df{r_R, 0.0f});
                r_th0 = r_d = r_beta = r_p = r_R = 0.0f;
            }
        }
        if (dead) break;
        // deterministic warp reduction of the parameter sums (double-single butterfly)
        df acc[5] = {acc_beta, acc_p, acc_th0, acc_d, acc_R};
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
                A.ginit[2 * r] = bf * GV0;
                A.ginit[2 * r + 1] = Ga0;
            }
        }
    }
    if (BULK) {
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

size_t alif_bwd_smem_bytes() {
    using namespace bwd;
    return (size_t)WARPS * NSTAGE * MAXARR * WIN * 4 + (size_t)WARPS * NSTAGE * 8;
}

int launch_alif_backward(long long B, long long N, long long T, const float *I,
                         const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                         const AlifState *ckpt, const float *gS, const float *gV, const float *ga,
                         const float *gfin, float slope, float *gI, float *ginit, float *part,
                         int *status, cudaStream_t stream) {
    using namespace bwd;
    Args A;
    A.rows = B * N;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + WIN - 1) / WIN;
    A.nwin = A.nckpt;
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
    A.narr = 2 + (gV ? 1 : 0) + (ga ? 1 : 0);
    if (g_sm_count_bwd == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count_bwd, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count_bwd <= 0) g_sm_count_bwd = 1;
    }
    auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    const bool bulk = (T % 4 == 0) && a16(I) && a16(gS) && (!gV || a16(gV)) && (!ga || a16(ga));
    const size_t smem = alif_bwd_smem_bytes();
    const long long need = (A.rows + WARPS - 1) / WARPS;
    static int occ[2] = {0, 0};
    const void *fn = bulk ? (const void *)bwd_kernel<true> : (const void *)bwd_kernel<false>;
    if (occ[bulk] == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, WARPS * 32, smem);
        occ[bulk] = n > 0 ? n : 1;
    }
    const long long cap = (long long)g_sm_count_bwd * occ[bulk];
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return 0;
    if (bulk)
        bwd_kernel<true><<<grid, WARPS * 32, smem, stream>>>(A);
    else
        bwd_kernel<false><<<grid, WARPS * 32, smem, stream>>>(A);
    return (int)cudaGetLastError();
}

}  // namespace alif
