// dL/dtau_mem of the rows whose membrane decays fast (beta < 1/2), completing the detached backward
// (Supplementary, "Surrogate gradient", "Detaching gradients") for sm_103a.
//
// The warp-per-row backward sums the beta gradient of its fast-sigmoid, trace-free variants in a
// same-step form, sum_t (V[t] - R m I[t]) G_V[t] = beta sum_t (V[t-1] (1 - S[t-1]) - R m I[t]) G_V[t];
// for small beta the same-step terms cancel (V[t] is then close to R m I[t]).  This kernel recomputes
// the shifted form for the rows with beta < 1/2 and rewrites their g_tau_mem partial; every other
// row is left as it is (a warp whose 32 rows all have beta >= 1/2 reads their beta and moves on).
//
// One lane per row, a warp per 32 consecutive rows, windows of 256 steps (one checkpoint stride)
// from the last to the first:
//   pass 1 re-runs the window forward from its checkpoint in 16-step sub-blocks with the stored
//          spikes (Eqs 2, 4, 5) and records the state entering each sub-block (shared memory);
//   pass 2 takes the sub-blocks in reverse, recomputes their membranes in registers and runs
//          G_V[t] = sg[t] gS[t] + beta (1 - S[t]) G_V[t+1] step by step, summing
//          (V[t-1] (1 - S[t-1]) - R m I[t]) G_V[t].
// A sub-block without a reset forms its membranes from the exact powers (V[k] = beta^{k+1} v_in + L[k])
// and passes its end state on in double-single; after a reset the chain restarts from an exact 0.
// G_V's chain multiplies by the rounded beta, whose memory is short here (beta^16 < 2^-16).
// Currents and upstream gradients arrive as [32 rows x 32 steps] 2-D TMA boxes (128-byte swizzle).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "common.cuh"
#include "tmap.h"

namespace alif {
namespace btm {

constexpr int SB = 16;                  // steps per sub-block
constexpr int WINS = ALIF_CKPT_STEPS;   // steps per window (one checkpoint stride)
constexpr int NSB = WINS / SB;          // sub-blocks per window
constexpr int NST = 6;                  // ring slots
constexpr int BOX_BYTES = 32 * 32 * 4;  // 32 rows x 32 steps
// the ring, its barriers, the sub-block states (v, a, rem: 3 x [NSB][32]), alignment of the ring
constexpr int SMEM_BYTES = NST * BOX_BYTES + NST * 8 + 3 * NSB * 32 * 4 + 1024;
constexpr float BETA_MIN = 0.5f;        // rows below it are recomputed here
static_assert(WINS % 32 == 0 && SB == 16, "two sub-blocks per box, whole boxes per window");

struct Args {
    long long rows, N, T, nwords, nckpt, nwin, ngroups;
    const AlifNeuron *nrn;
    const uint32_t *spikes;
    const AlifState *ckpt, *init;
    const float *gfin;
    float slope;
    float *part;
    int *status;
};

// Admitted steps (bit k) of a sub-block entering with `rel` refractory steps, spikes `sb` and a
// refractory span of teff - 1 steps after each spike (Eq 4).
__device__ __forceinline__ unsigned admitted(int rel, unsigned sb, int teff) {
    unsigned mb = rel >= SB ? 0u : (0xFFFFu & ~((1u << rel) - 1u));
    for (unsigned sp = sb; sp; sp &= sp - 1u) {
        const int j = __ffs(sp) - 1;
        const int n = min(teff - 1, SB - 1 - j);
        mb &= ~(((1u << n) - 1u) << (j + 1));
    }
    return mb;
}

// This lane's 16 floats of box row `lane`, sub-block h (chunks 4h .. 4h + 3 under the swizzle).
__device__ __forceinline__ void load16(const float *row, int h, int sw, float (&x)[SB]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 u = *reinterpret_cast<const float4 *>(row + 4 * ((4 * h + q) ^ sw));
        x[4 * q] = u.x;
        x[4 * q + 1] = u.y;
        x[4 * q + 2] = u.z;
        x[4 * q + 3] = u.w;
    }
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

__global__ void __launch_bounds__(32) bwd_taumem_kernel(const __grid_constant__ CUtensorMap tmI,
                                                        const __grid_constant__ CUtensorMap tmS, const Args A) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 128-byte swizzle: 1024-aligned boxes
    float *ring = reinterpret_cast<float *>(sm);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NST * BOX_BYTES);
    float *sv = reinterpret_cast<float *>(sm + NST * BOX_BYTES + NST * 8);  // [NSB][32] v entering
    float *sa = sv + NSB * 32;                                               // [NSB][32] a entering
    int *srel = reinterpret_cast<int *>(sa + NSB * 32);                      // [NSB][32] rem entering
    const int lane = threadIdx.x;
    const long long ng = gridDim.x;
    const int T = (int)A.T;
    const int nwin = (int)A.nwin;

    // the next group, from g on, holding a row with beta < 1/2 (ngroups if none)
    auto next_group = [&](long long g) {
        for (; g < A.ngroups; g += ng) {
            const long long r = g * 32 + lane;
            const bool need = r < A.rows && A.nrn[r % A.N].beta_hi < BETA_MIN;
            if (__any_sync(FULL, need)) break;
        }
        return g;
    };
    const long long g_first = next_group(blockIdx.x);
    if (g_first >= A.ngroups) return;  // warp-uniform: nothing to recompute here

    // ---- TMA producer (lane 0 issues; every lane tracks the cursor).  Per window, newest first:
    // its currents' boxes b = 0 .. nb-1 (pass 1), then (currents, gradients) of boxes nb-1 .. 0.
    long long p_g = g_first;
    int p_wi = nwin - 1, p_it = 0;
    unsigned issued = 0, consumed = 0;
    if (lane == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    auto boxes = [&](int wi) {  // boxes of window wi holding steps < T
        const int left = T - wi * WINS;
        return left >= WINS ? WINS / 32 : (left + 31) / 32;
    };
    auto issue = [&]() {
        while (p_g < A.ngroups && issued - consumed < (unsigned)NST) {
            const int nb = boxes(p_wi);
            if (lane == 0) {
                const int st = issued % NST;
                int b, arr;
                if (p_it < nb) {
                    b = p_it;
                    arr = 0;
                } else {
                    const int j = p_it - nb;
                    b = nb - 1 - (j >> 1);
                    arr = j & 1;
                }
                mbar_arrive_expect_tx(&bars[st], BOX_BYTES);
                tma_load_2d_u(smem_u32(ring) + st * BOX_BYTES, arr ? &tmS : &tmI, p_wi * WINS + 32 * b,
                              (int)(p_g * 32), smem_u32(&bars[st]));
            }
            ++issued;
            if (++p_it == 3 * nb) {
                p_it = 0;
                if (--p_wi < 0) {
                    p_wi = nwin - 1;
                    p_g = next_group(p_g + ng);
                }
            }
        }
    };
    issue();
    // the box `ahead` places after the next one to be released: waits for it, returns this lane's row
    auto take = [&](unsigned ahead, const float *&row) -> bool {
        const unsigned k = consumed + ahead;
        const int st = k % NST;
        if (!mbar_wait_bounded(&bars[st], (k / NST) & 1u)) {
            report_timeout(A.status);
            return false;
        }
        row = ring + st * (BOX_BYTES / 4) + lane * 32;
        return true;
    };
    auto release = [&](int n) {  // the n oldest boxes are read
        __syncwarp();
        fence_proxy_async_smem();
        consumed += n;
        issue();
    };

    const int sw = lane & 7;
    bool dead = false;
    for (long long g = g_first; g < A.ngroups && !dead; g = next_group(g + ng)) {
        const long long r = g * 32 + lane;
        const bool live = r < A.rows;
        const AlifNeuron nr = A.nrn[(live ? r : g * 32) % A.N];
        const bool mine = live && nr.beta_hi < BETA_MIN;  // this lane's row is recomputed
        const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo};
        const float bf = nr.beta_hi, c = nr.c_hi, d = nr.d, th0 = nr.theta0, Rr = nr.R, pf = nr.p_hi;
        const float slope = A.slope;
        const int teff = nr.teff;
        float Bk[SB];  // beta^(k+1)
        df B16, P16;   // beta^16, p^16
        {
            P16 = df_pow(p, SB);
            df q{1.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < SB; ++k) {
                q = df_mul(q, beta);
                Bk[k] = q.hi;
            }
            B16 = q;
        }
        const uint32_t *words = A.spikes + (live ? r : 0) * A.nwords;
        float GVn = (A.gfin && live) ? A.gfin[2 * r] : 0.0f;  // dL/dV of the step after the current one
        df acc{0.0f, 0.0f};

        for (int wi = nwin - 1; wi >= 0 && !dead; --wi) {
            const int w = wi * WINS;
            const int cnt = T - w >= WINS ? WINS : T - w;
            const int nb = (cnt + 31) / 32;
            const bool last_window = wi == nwin - 1;
            AlifState cs{0.0f, 0.0f, 0};
            if (live) cs = A.ckpt ? A.ckpt[r * A.nckpt + wi] : (A.init ? A.init[r] : cs);
            // ---- pass 1: the window forward from its checkpoint, recording each sub-block's entry
            // (membrane and adaptation carried in double-single between sub-blocks)
            {
                int rel = cs.rem > 0 ? cs.rem : 0;
                df Vd{rel > 0 ? 0.0f : cs.v, 0.0f};
                df aw{cs.a, 0.0f};
                for (int b = 0; b < nb; ++b) {
                    const float *row;
                    if (!take(0, row)) {
                        dead = true;
                        break;
                    }
                    const uint32_t wd = live ? __ldg(words + (w >> 5) + b) : 0u;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int s = 2 * b + h;
                        if (16 * s >= cnt) break;  // warp-uniform
                        sv[s * 32 + lane] = Vd.hi;
                        sa[s * 32 + lane] = aw.hi;
                        srel[s * 32 + lane] = rel;
                        float x[SB];
                        load16(row, h, sw, x);
                        const unsigned sb = (wd >> (16 * h)) & 0xFFFFu;
                        const unsigned mb = admitted(rel, sb, teff);
                        float L = 0.0f, as = 0.0f;
#pragma unroll
                        for (int k = 0; k < SB; ++k) {
                            const float cx = ((mb >> k) & 1u) ? c * x[k] : 0.0f;
                            const bool reset = k > 0 && ((sb >> (k - 1)) & 1u);
                            L = fmaf(reset ? 0.0f : bf, L, cx);
                            as = fmaf(pf, as, ((sb >> k) & 1u) ? 1.0f : 0.0f);  // the spikes' decayed units
                        }
                        if (sb == 0u)
                            Vd = df_fma_f(B16, Vd, L);
                        else
                            Vd = ((sb >> 15) & 1u) ? df{0.0f, 0.0f} : df{L, 0.0f};
                        {
                            const df an = df_mul(aw, P16);
                            const df ss = two_sum(an.hi, as);
                            aw = quick_two_sum(ss.hi, ss.lo + an.lo);
                        }
                        const int jl = sb ? 31 - __clz(sb) : -1;  // last spike of the sub-block
                        rel = sb ? max(jl + teff - SB, 0) : max(rel - SB, 0);
                    }
                    release(1);
                }
                if (dead) break;
            }

            // ---- pass 2: sub-blocks in reverse: recompute, then G_V and the beta sum
            float sbeta = 0.0f;
            for (int b = nb - 1; b >= 0; --b) {
                const float *rowI, *rowG;
                if (!take(0, rowI) || !take(1, rowG)) {
                    dead = true;
                    break;
                }
                const uint32_t wd = live ? __ldg(words + (w >> 5) + b) : 0u;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int h = 1 - hh;
                    const int s = 2 * b + h;
                    const int cs_ = cnt - 16 * s;  // steps of this sub-block (<= 0: none)
                    if (cs_ <= 0) continue;        // warp-uniform
                    const bool tail = cs_ < SB;    // the row's last, partial sub-block
                    const bool row_end = last_window && 16 * s + SB >= cnt;
                    float x[SB], gs[SB];
                    load16(rowI, h, sw, x);
                    load16(rowG, h, sw, gs);
                    const float v0 = sv[s * 32 + lane], a0 = sa[s * 32 + lane];
                    const int rel = srel[s * 32 + lane];
                    const unsigned sb = (wd >> (16 * h)) & 0xFFFFu;
                    const unsigned mb = admitted(rel, sb, teff);
                    float V[SB], a[SB];
                    {
                        const int fr = sb ? __ffs(sb) : SB;  // first step after a reset
                        float L = 0.0f, ak = a0;
#pragma unroll
                        for (int k = 0; k < SB; ++k) {
                            const float cx = ((mb >> k) & 1u) ? c * x[k] : 0.0f;
                            const bool reset = k > 0 && ((sb >> (k - 1)) & 1u);
                            L = fmaf(reset ? 0.0f : bf, L, cx);
                            V[k] = k < fr ? fmaf(Bk[k], v0, L) : L;
                            a[k] = ak;
                            ak = fmaf(pf, ak, ((sb >> k) & 1u) ? 1.0f : 0.0f);
                        }
                    }
#pragma unroll
                    for (int k = SB - 1; k >= 0; --k) {
                        const bool valid = !tail || k < cs_;
                        const float u = V[k] - fmaf(d, a[k], th0);
                        const float den = fmaf(slope, fabsf(u), 1.0f);
                        const float sgv = valid ? gs[k] * __fdividef(1.0f, den * den) : 0.0f;
                        const bool spk = (sb >> k) & 1u;
                        // into the next step: beta (1 - S), or (1 - S) at the row's last step
                        const bool lastk = row_end && k == cs_ - 1;
                        const float F = spk ? 0.0f : (lastk ? 1.0f : bf);
                        const float GV = valid ? fmaf(F, GVn, sgv) : GVn;
                        const float xi = ((mb >> k) & 1u) ? x[k] : 0.0f;
                        const float vent = k == 0 ? v0 : (((sb >> (k - 1)) & 1u) ? 0.0f : V[k - 1]);
                        if (valid) sbeta = fmaf(fmaf(-Rr, xi, vent), GV, sbeta);
                        GVn = GV;
                    }
                }
                release(2);
            }
            if (dead) break;
            acc = df_add(acc, df{sbeta, 0.0f});
        }
        if (dead) break;
        if (mine) {
            const df gtm = df_mul_f(acc, nr.dbeta_dtau);
            float *o = A.part + r * (2 * ALIF_NUM_PARAM_GRADS);
            o[2 * ALIF_G_TAU_MEM] = gtm.hi;
            o[2 * ALIF_G_TAU_MEM + 1] = gtm.lo;
        }
    }

    // never leave a copy in flight into this CTA's shared memory
    while (consumed < issued) {
        if (!mbar_wait_bounded(&bars[consumed % NST], (consumed / NST) & 1u)) {
            report_timeout(A.status);
            break;
        }
        ++consumed;
    }
}

}  // namespace btm

static int g_sm_count_btm = 0;

// Follow-up of the warp-per-row backward's same-step variants (fast sigmoid, no trace gradients, TMA
// staging): rewrites g_tau_mem of the rows with beta < 1/2 in `part`.  The caller has checked the
// TMA conditions (T a multiple of 16, I and dL/dS 16-byte aligned).
int launch_alif_backward_taumem(long long rows, long long N, long long T, const float *I, const AlifNeuron *nrn,
                                const uint32_t *spikes, const AlifState *ckpt, const AlifState *init,
                                const float *gS, const float *gfin, float slope, float *part, int *status,
                                cudaStream_t stream) {
    using namespace btm;
    CUtensorMap m[2];
    memset(m, 0, sizeof m);
    if (make_rowmajor_map(&m[0], I, rows, T) != 0 || make_rowmajor_map(&m[1], gS, rows, T) != 0)
        return (int)cudaErrorInvalidValue;
    Args A;
    memset(&A, 0, sizeof A);
    A.rows = rows;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS;
    A.nwin = (T + WINS - 1) / WINS;
    A.ngroups = (rows + 31) / 32;
    A.nrn = nrn;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.init = init;
    A.gfin = gfin;
    A.slope = slope;
    A.part = part;
    A.status = status;
    if (g_sm_count_btm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count_btm, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count_btm <= 0) g_sm_count_btm = 1;
    }
    static int occ = 0;
    const void *fn = (const void *)bwd_taumem_kernel;
    if (occ == 0) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32, SMEM_BYTES);
        occ = n > 0 ? n : 1;
    }
    const long long cap = (long long)g_sm_count_btm * occ;
    const int grid = (int)(A.ngroups < cap ? A.ngroups : cap);
    if (grid <= 0) return 0;
    void *args[] = {&m[0], &m[1], &A};
    return (int)cudaLaunchKernel(fn, dim3(grid), dim3(32), args, SMEM_BYTES, stream);
}

}  // namespace alif
