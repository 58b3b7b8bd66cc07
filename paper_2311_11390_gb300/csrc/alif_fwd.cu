// ARP-blocked ALIF forward (Section 3, Props 1-5) for sm_103a.
//
// One warp simulates one neuron row at a time and walks time in windows of
// WIN = 256 steps, lane L holding steps 8L..8L+7 of the window.  A window is
// resolved in "rounds":
//   1. the no-reset membrane of Prop 1 over the admitted part of the window,
//      V~[t] = beta^{t+1} v_in + sum_{j<=t} beta^{t-j} (1-beta) R I[j],
//      is a decayed prefix scan (8-step in-lane recurrence + 5-level shuffle
//      scan across lanes);
//   2. the adaptive threshold is theta0 + d p^t a_w (Prop 5, no spike yet);
//   3. the first crossing V~ > theta (Props 2 and Eq 9: only the first faulty
//      spike is real) is found with a warp ballot and __ffs;
//   4. after a spike at tau the membrane is reset (Prop 4) and input is masked
//      until tau + T_eff (Prop 3), so the next round rescans from there with a
//      zero start; the adaptation restarts from a[tau+1] = p a[tau] + 1 (Prop 5).
// A window without spikes therefore costs one round however many T_R-blocks
// it spans; a window with k spikes costs k+1 rounds (never more than the
// ceil(256/T_R)+1 blocks the fixed-block schedule would visit).
//
// Exactness of the spike decisions: the FP32 margin M = V~ - theta comes with
// an error bound G (guard * (|V~| + theta + R max|I|)).  |M| <= G is
// re-decided in double-single arithmetic from an exact anchor (the last reset,
// where V is exactly 0, or the last re-decided step), re-reading the inputs
// since the anchor from global memory.  Decisions then agree with the FP64
// standard model except for margins ~1e-13.
#include "common.cuh"

namespace alif {
namespace fwd {

constexpr int E = 8;           // steps per lane
constexpr int WIN = 32 * E;    // window = checkpoint stride
constexpr int NSTAGE = 4;      // bulk-copy ring depth per warp
constexpr int WARPS = 4;       // warps per CTA
constexpr int SMEM_PER_WARP = NSTAGE * WIN * 4 + NSTAGE * 8 + 2 * (WIN + 1) * 4 + 8;  // ring, barriers, p^j
static_assert(WIN == ALIF_CKPT_STEPS, "window must equal the checkpoint stride");

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
};

// Inclusive decayed prefix scan over the warp's 256 steps:
// v[t] <- sum_{j<=t} dec^{t-j} v[j].  Blm[l] = dec^(8*2^l) on lanes >= 2^l and 0
// below (so no per-level predicate), bk1m[k] = dec^(k+1) on lanes > 0, 0 on lane 0.
__device__ __forceinline__ void decay_scan(float (&v)[E], float dec, const float (&Blm)[5],
                                           const float (&bk1m)[E]) {
#pragma unroll
    for (int k = 1; k < E; ++k) v[k] = fmaf(dec, v[k - 1], v[k]);
    float tot = v[E - 1];
#pragma unroll
    for (int l = 0; l < 5; ++l) tot = fmaf(Blm[l], __shfl_up_sync(FULL, tot, 1 << l), tot);
    const float P = __shfl_up_sync(FULL, tot, 1);
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = fmaf(bk1m[k], P, v[k]);
}

// Exact (double-single) membrane at global step t, from the anchor
// "V entering step anc_t equals anc_v" with no spike or mask in [anc_t, t]:
//   V[t] = beta^{t-anc_t+1} anc_v + sum_{j=anc_t}^{t} beta^{t-j} c I[j].
// Warp-cooperative: each lane takes a contiguous piece (Horner), pieces are
// scaled to t and summed with a butterfly (same result in every lane).
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
    for (long long j = lo; j < hi; ++j) h = df_add(df_mul(h, beta), df_mul_f(c, __ldg(Irow + j)));
    if (hi > lo) h = df_mul(h, df_pow(beta, t - (hi - 1)));
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const df o{__shfl_xor_sync(FULL, h.hi, off), __shfl_xor_sync(FULL, h.lo, off)};
        h = df_add(h, o);
    }
    return df_add(h, df_mul(df_pow(beta, n), df{anc_hi, anc_lo}));
}

template <bool BULK, bool VTR, bool ATR>
__global__ void __launch_bounds__(WARPS * 32, 4) fwd_kernel(const Args A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wsm = smem + warp * SMEM_PER_WARP;
    float *ring = reinterpret_cast<float *>(wsm);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + NSTAGE * WIN * 4);
    float *pdh = reinterpret_cast<float *>(wsm + NSTAGE * WIN * 4 + NSTAGE * 8);  // p^j hi, j=0..WIN
    float *pdl = pdh + (WIN + 1);                                                  // p^j lo
    const long long gw = (long long)blockIdx.x * WARPS + warp;
    const long long nw = (long long)gridDim.x * WARPS;
    if (gw >= A.rows) return;  // warps are independent: no block-level barrier below

    // ---- bulk-copy producer (lane 0 issues; every lane tracks the cursor)
    long long p_row = gw;
    int p_wi = 0;
    const int nwin = (int)A.nwin;
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
            if (lane == 0) {
                const int st = issued % NSTAGE;
                const long long w0 = (long long)p_wi * WIN;
                const long long left = A.T - w0;
                const uint32_t bytes = (uint32_t)((left < WIN ? left : WIN) * 4);
                mbar_arrive_expect_tx(&bars[st], bytes);
                bulk_g2s_stream(ring + st * WIN, A.I + p_row * A.T + w0, bytes, &bars[st], pol);
            }
            ++issued;
            if (++p_wi == nwin) {
                p_wi = 0;
                p_row += nw;
            }
        }
    };
    if (BULK) issue();

    bool dead = false;
    unsigned long long n_exact = 0, n_exact_spk = 0, n_rows = 0;
    const int t0 = 8 * lane;

    for (long long r = gw; r < A.rows && !dead; r += nw) {
        const AlifNeuron nr = A.nrn[r % A.N];
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        const float *Irow = A.I + r * A.T;

        // Per-lane decay tables rounded once from double-single powers, and the
        // warp's table of p^j (j = 0..256) as double-single pairs.
        float dPw[E], Pw[E], bk1[E], bk1u[E], Bl[5];
        float B0;  // beta^{8L}: V at window step t is beta^{t+1} v_in = bk1u[k] (B0 v_in)
        {
            df q = df_pow(p, t0), u = beta;
            B0 = df_pow(beta, t0).hi;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                Pw[k] = q.hi;           // p^t
                dPw[k] = nr.d * q.hi;   // d p^t
                bk1[k] = u.hi;          // beta^{k+1}
                bk1u[k] = u.hi;
                pdh[t0 + k] = q.hi;
                pdl[t0 + k] = q.lo;
                q = df_mul(q, p);
                u = df_mul(u, beta);
            }
            if (lane == 31) {
                pdh[WIN] = q.hi;
                pdl[WIN] = q.lo;
            }
            df b8 = df_pow(beta, 8);
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                Bl[l] = lane >= (1 << l) ? b8.hi : 0.0f;
                b8 = df_mul(b8, b8);
            }
#pragma unroll
            for (int k = 0; k < E; ++k)
                if (lane == 0) bk1[k] = 0.0f;
        }
        __syncwarp();
        auto pdf = [&](int j) { return df{pdh[j], pdl[j]}; };

        // ---- state entering the row
        float Vin;
        df aw;
        long long res, anc_t;
        df anc_v;
        {
            AlifState s0{0.0f, 0.0f, 0};
            if (A.init) s0 = A.init[r];
            const int rem = s0.rem > 0 ? s0.rem : 0;
            Vin = rem > 0 ? 0.0f : s0.v;
            aw = df{s0.a, 0.0f};
            res = rem;
            anc_t = rem;
            anc_v = df{Vin, 0.0f};
        }
        float mxr = 0.0f;

        for (int wi = 0; wi < nwin; ++wi) {
            const long long w = (long long)wi * WIN;
            const int cnt = (int)(A.T - w < WIN ? A.T - w : WIN);
            float x[E];
            if (BULK) {
                const int st = consumed % NSTAGE;
                const uint32_t par = (consumed / NSTAGE) & 1u;
                if (!mbar_wait_bounded(&bars[st], par)) {
                    report_timeout(A.status);
                    dead = true;
                    break;
                }
                const float4 *src = reinterpret_cast<const float4 *>(ring + st * WIN + t0);
                const float4 u0 = src[0], u1 = src[1];
                x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
                __syncwarp();
                fence_proxy_async_smem();
                ++consumed;
                issue();
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) x[k] = (t0 + k < cnt) ? __ldg(Irow + w + t0 + k) : 0.0f;
            }
            if (cnt < WIN) {
#pragma unroll
                for (int k = 0; k < E; ++k)
                    if (t0 + k >= cnt) x[k] = 0.0f;
            }

            if (A.ckpt && lane == 0) {
                AlifState cs;
                cs.v = Vin;
                cs.a = aw.hi;
                cs.rem = (int)(res - w > 0 ? res - w : 0);
                A.ckpt[r * A.nckpt + wi] = cs;
            }

            // Scale of the error bound.  V is a convex combination of v_in and
            // R I[j], so |V| <= max(|v_in|, R max|I|); errors carried from earlier
            // windows are bounded through the row's running max of |I|.
            float mx = 0.0f;
#pragma unroll
            for (int k = 0; k < E; ++k) mx = fmaxf(mx, fabsf(x[k]));
#pragma unroll
            for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
            mxr = fmaxf(mx, mxr);
            const float Rmx = nr.R * mx, gs = nr.R * mxr;

            const long long s1l = res - w;
            const int s1 = (int)(s1l <= 0 ? 0 : (s1l >= cnt ? cnt : s1l));
            float V[E], Z[E], vt[E], a_el[E];
            // ---- round 1: no spike since the window start (a = p^t a_w)
            float G = nr.guard * (fmaxf(fabsf(Vin), Rmx) + nr.theta0 + nr.d * aw.hi + gs);
            {
                float q[E];
                if (s1 == 0) {
#pragma unroll
                    for (int k = 0; k < E; ++k) q[k] = nr.c_hi * x[k];
                } else {
#pragma unroll
                    for (int k = 0; k < E; ++k) q[k] = (t0 + k >= s1) ? nr.c_hi * x[k] : 0.0f;
                }
                decay_scan(q, beta.hi, Bl, bk1);
                const float thG = nr.theta0 - G;
                const float BV = B0 * Vin;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    V[k] = fmaf(bk1u[k], BV, q[k]);
                    Z[k] = V[k] - fmaf(dPw[k], aw.hi, thG);  // V - theta + G
                    if (VTR) vt[k] = V[k];
                    if (ATR) a_el[k] = Pw[k] * aw.hi;
                }
            }
            bool any;
            if (s1 == 0 && cnt == WIN) {  // common case: every step of the window is eligible
                const float zm = fmaxf(fmaxf(fmaxf(Z[0], Z[1]), fmaxf(Z[2], Z[3])),
                                       fmaxf(fmaxf(Z[4], Z[5]), fmaxf(Z[6], Z[7])));
                any = __any_sync(FULL, zm >= 0.0f);
            } else {
                bool mine = false;
#pragma unroll
                for (int k = 0; k < E; ++k) mine |= (t0 + k >= s1) && (t0 + k < cnt) && (Z[k] >= 0.0f);
                any = __any_sync(FULL, mine);
            }

            uint32_t sword = 0;
            int last_tau = -1, s2 = 0, aanc_rel = 0;
            df aanc = aw, A1{0.0f, 0.0f};
            if (any) {
                // ---- resolve crossings in order: exact re-decision inside the
                // error band, spike, reset + ARP skip, rescan
                int search = s1;
                while (search < cnt) {
                    unsigned fm = 0;
#pragma unroll
                    for (int k = 0; k < E; ++k)
                        fm |= (unsigned)((t0 + k >= search) && (t0 + k < cnt) && (Z[k] >= 0.0f)) << k;
                    const unsigned bal = __ballot_sync(FULL, fm != 0u);
                    if (bal == 0u) break;
                    const int Lf = __ffs(bal) - 1;
                    const int kf = __ffs(__shfl_sync(FULL, fm, Lf)) - 1;
                    float zsel = Z[0];
#pragma unroll
                    for (int k = 1; k < E; ++k)
                        if (k == kf) zsel = Z[k];
                    const float zf = __shfl_sync(FULL, zsel, Lf);
                    const int tf = 8 * Lf + kf;
                    if (!(zf > 2.0f * G)) {
                        // margin within the FP32 error bound: decide exactly
                        ++n_exact;
                        const long long tg = w + tf;
                        const df Vx = exact_membrane(Irow, anc_t, anc_v.hi, anc_v.lo, tg, nr.beta_hi,
                                                     nr.beta_lo, nr.c_hi, nr.c_lo, lane);
                        const df ax = df_mul(pdf(tf - aanc_rel), aanc);
                        const df thx = df_add(df_mul_f(ax, nr.d), df{nr.theta0, 0.0f});
                        if (df_cmp(Vx, thx) <= 0) {
                            anc_t = tg + 1;  // exact V is now known entering tg + 1
                            anc_v = Vx;
                            search = tf + 1;
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
                    res = w + tau + nr.teff;  // input admitted again from here (Eq 4)
                    anc_t = res;              // V is exactly 0 entering res
                    anc_v = df{0.0f, 0.0f};
                    s2 = tau + nr.teff;
                    // a[t] = p^{t-tau-1} A1 for t > tau, p^e assembled from lane powers
                    float pe[E];
                    {
                        const int t1 = tau + 1, Lq = t1 >> 3, kq = t1 & 7;
                        const float vA = __shfl_sync(FULL, Pw[0], (lane - Lq) & 31);
                        const float vB = __shfl_sync(FULL, Pw[0], (lane - Lq - 1) & 31);
#pragma unroll
                        for (int k = 0; k < E; ++k) {
                            const bool up = k >= kq;
                            pe[k] = (up ? vA : vB) * pdh[up ? k - kq : 8 + k - kq];
                            if (ATR && t0 + k > tau) a_el[k] = pe[k] * A1.hi;
                            if (VTR && t0 + k > tau) vt[k] = 0.0f;
                        }
                    }
                    if (s2 >= cnt) break;
                    {
                        G = nr.guard * (Rmx + nr.theta0 + nr.d * A1.hi + gs);
                        float q[E];
#pragma unroll
                        for (int k = 0; k < E; ++k) q[k] = (t0 + k >= s2) ? nr.c_hi * x[k] : 0.0f;
                        decay_scan(q, beta.hi, Bl, bk1);
                        const float dA = nr.d * A1.hi, thG = nr.theta0 - G;
#pragma unroll
                        for (int k = 0; k < E; ++k) {
                            V[k] = q[k];
                            Z[k] = V[k] - fmaf(dA, pe[k], thG);
                            if (VTR && t0 + k >= s2) vt[k] = V[k];
                        }
                    }
                    search = s2;
                }
            }

            // ---- outputs of the window
            if (lane < E) {
                const long long widx = (long long)wi * E + lane;
                if (widx < A.nwords) A.spikes[r * A.nwords + widx] = sword;
            }
            if (VTR || ATR) {
                float *vo = VTR ? A.vtr + r * A.T + w + t0 : nullptr;
                float *ao = ATR ? A.atr + r * A.T + w + t0 : nullptr;
                if (BULK && t0 + E <= cnt) {
                    if (VTR) {
                        reinterpret_cast<float4 *>(vo)[0] = make_float4(vt[0], vt[1], vt[2], vt[3]);
                        reinterpret_cast<float4 *>(vo)[1] = make_float4(vt[4], vt[5], vt[6], vt[7]);
                    }
                    if (ATR) {
                        reinterpret_cast<float4 *>(ao)[0] = make_float4(a_el[0], a_el[1], a_el[2], a_el[3]);
                        reinterpret_cast<float4 *>(ao)[1] = make_float4(a_el[4], a_el[5], a_el[6], a_el[7]);
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
                const int tl = cnt - 1, kl = tl & 7;
                float mine = V[E - 1];
                if (cnt < WIN) {
#pragma unroll
                    for (int k = 0; k < E - 1; ++k)
                        if (k == kl) mine = V[k];
                }
                Vnext = __shfl_sync(FULL, mine, tl >> 3);
                if (last_tau >= 0 && s2 >= cnt) Vnext = 0.0f;  // still reset / refractory
            }
            if (last_tau < 0)
                aw = df_mul(aw, pdf(cnt));
            else
                aw = df_mul(pdf(cnt - last_tau - 1), A1);
            Vin = Vnext;
        }
        if (dead) break;
        if (A.fin && lane == 0) {
            AlifState fs;
            fs.v = Vin;
            fs.a = aw.hi;
            fs.rem = (int)(res - A.T > 0 ? res - A.T : 0);
            A.fin[r] = fs;
        }
        ++n_rows;
        __syncwarp();  // the p^j table is rewritten for the next row
    }

    if (BULK) {  // never leave a copy in flight into this CTA's shared memory
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

}  // namespace fwd

// --------------------------------------------------------------- launcher
static int g_sm_count = 0;

int launch_alif_forward(long long B, long long N, long long T, const float *I,
                        const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                        float *vtr, float *atr, AlifState *ckpt, AlifState *fin,
                        unsigned long long *counters, int *status, cudaStream_t stream) {
    using namespace fwd;
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
    auto aligned16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    const bool bulk = (T % 4 == 0) && aligned16(I) && (!vtr || aligned16(vtr)) && (!atr || aligned16(atr));
    const size_t smem = (size_t)WARPS * SMEM_PER_WARP;
    const long long need = (A.rows + WARPS - 1) / WARPS;
    const int sel = (bulk ? 4 : 0) | (vtr ? 2 : 0) | (atr ? 1 : 0);
    // one resident wave: CTAs per SM from the occupancy of the selected variant
    static int occ[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (occ[sel] == 0) {
        const void *fn = nullptr;
        switch (sel) {
            case 0: fn = (const void *)fwd_kernel<false, false, false>; break;
            case 1: fn = (const void *)fwd_kernel<false, false, true>; break;
            case 2: fn = (const void *)fwd_kernel<false, true, false>; break;
            case 3: fn = (const void *)fwd_kernel<false, true, true>; break;
            case 4: fn = (const void *)fwd_kernel<true, false, false>; break;
            case 5: fn = (const void *)fwd_kernel<true, false, true>; break;
            case 6: fn = (const void *)fwd_kernel<true, true, false>; break;
            default: fn = (const void *)fwd_kernel<true, true, true>; break;
        }
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, WARPS * 32, smem);
        occ[sel] = n > 0 ? n : 1;
    }
    const long long cap = (long long)g_sm_count * occ[sel];
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return 0;
#define ALIF_FWD_LAUNCH(BK, VT, AT) fwd_kernel<BK, VT, AT><<<grid, WARPS * 32, smem, stream>>>(A)
    switch (sel) {
        case 0: ALIF_FWD_LAUNCH(false, false, false); break;
        case 1: ALIF_FWD_LAUNCH(false, false, true); break;
        case 2: ALIF_FWD_LAUNCH(false, true, false); break;
        case 3: ALIF_FWD_LAUNCH(false, true, true); break;
        case 4: ALIF_FWD_LAUNCH(true, false, false); break;
        case 5: ALIF_FWD_LAUNCH(true, false, true); break;
        case 6: ALIF_FWD_LAUNCH(true, true, false); break;
        default: ALIF_FWD_LAUNCH(true, true, true); break;
    }
#undef ALIF_FWD_LAUNCH
    return (int)cudaGetLastError();
}

}  // namespace alif
