// Recurrent ALIF layer with transmission latency D = T_R (sm_103a).
//
// Section 2 lets the input current of Eq 3 carry a recurrent term
// sum_j W_rec[i][j] S_j[t - D] and assumes the latency D equals the ARP, T_R.
// Prop 3 is what makes that useful: the recurrent current of Block n+1 is
// fixed by the spikes of Block n, so a whole population advances T_R steps
// between two exchanges of spikes instead of one.
//
// One batch element is one thread-block cluster of G CTAs (G <= 8), each CTA
// owning up to 1024 consecutive neurons, one thread per neuron.  Per Block of
// T_R steps:
//   1. after a cluster barrier, every CTA reads the previous Block's spikes of
//      all N neurons from the G CTAs' shared memory (distributed shared
//      memory) -- at most one spike per neuron and Block, since the ARP
//      (T_eff = max(T_R, 2) >= T_R) allows no second one -- and lists them;
//   2. each thread adds W_rec[i][j] for every listed spike (j, t) into its
//      column of a [T_R x neurons] double-single shared accumulator, started
//      from the feedforward current I_ff[t] of its row (W_rec is stored
//      transposed, so a warp reads 128 contiguous bytes per spike).  The
//      weights of up to WCH spikes are copied into shared memory together
//      (cp.async, one round trip), and the feedforward current of Block n+1
//      is copied into a second accumulator while Block n is resolved, so
//      neither HBM read sits on the Block's critical path;
//   3. each thread steps its neuron through the Block (Eqs 1-5, state form)
//      with the current, V and a in double-single, so that every spike
//      decision is the one exact arithmetic takes (a flip needs a margin near
//      1e-12); it publishes the step of its spike (or none) for the next Block.
// The total current I_ff + I_rec, rounded to FP32, is written out for the backward, with the
// spike words, the checkpoints every ALIF_CKPT_STEPS steps and the final state
// in the layouts of alif_forward.  Every CTA of a cluster runs the same number
// of cluster barriers, and the last one keeps every CTA's shared memory alive
// until no other CTA reads it.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace alif {
namespace rec {

constexpr int MAX_G = 8;           // portable cluster size
constexpr int MAX_PER = 1024;      // neurons per CTA
constexpr int NO_SPIKE = -1;
constexpr int MAX_WCH = 32;        // recurrent weights copied together

struct Args {
    long long B, N, T, nwords, nckpt;
    int TR, G, per;
    int nbuf;  // 2: the next Block's current is prefetched into a second accumulator
    int wch;   // spikes whose weights are copied into shared memory together
    const float *Iff;
    const float *Wt;  // [N pre, N post]
    const AlifNeuron *nrn;
    const AlifState *init;
    float *Iout;
    uint32_t *spikes;
    AlifState *ckpt, *fin;
};

// acc [nbuf][TR][per + 1] (rows padded by one float, so that a warp reading or writing 32
// rows' chunks through it spreads over the banks), acl [TR][per], wbuf [wch][per] (floats);
// spk [2][per]; list [N]; wsum [64]
__host__ __device__ constexpr size_t smem_bytes(int TR, int per, long long N, int nbuf, int wch) {
    return (size_t)nbuf * TR * (per + 1) * 4 + (size_t)TR * per * 4 + (size_t)wch * per * 4 + (size_t)2 * per * 4 +
           (size_t)N * 4 + 64 * 4;
}

// 4-byte asynchronous global -> shared copy (completion tracked by cp.async groups)
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// b v + x for double-single b, v, x: the product of the high parts split exactly (FMA), the
// low-order terms added once (relative error about 2^-46); a shorter dependent chain than a
// double-single product followed by a double-single sum
__device__ __forceinline__ df df_axpy(df b, df v, df x) {
    const float p = b.hi * v.hi;
    const float e = fmaf(b.hi, v.hi, -p);
    const df s = two_sum(p, x.hi);
    float lo = e + s.lo;
    lo = fmaf(b.hi, v.lo, lo);
    lo = fmaf(b.lo, v.hi, lo);
    lo += x.lo;
    return quick_two_sum(s.hi, lo);
}

// MAXT: the CTA size the register budget is sized for (256: up to 255 registers a thread, for
// clusters of at most 256 neurons per CTA; 1024 otherwise)
template <int MAXT>
__global__ void __launch_bounds__(MAXT) rec_fwd_kernel(const Args A) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int per = A.per, TR = A.TR, G = A.G, nbuf = A.nbuf, wch = A.wch;
    const int ld = per + 1;                                                          // acc row stride
    float *acc = reinterpret_cast<float *>(smem);                                   // [nbuf][TR][ld] hi
    float *acl = acc + (size_t)nbuf * TR * ld;                                       // [TR][per] lo
    float *wbuf = acl + (size_t)TR * per;                                            // [wch][per] weights
    int *spk = reinterpret_cast<int *>(wbuf + (size_t)wch * per);                    // [2][per]
    uint32_t *list = reinterpret_cast<uint32_t *>(spk + 2 * per);                    // [N] (j << 10) | t
    int *wsum = reinterpret_cast<int *>(list + A.N);                                 // [32] + total
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = (per + 31) >> 5;
    const int rank = (int)cl.block_rank();
    const long long b = blockIdx.x / G;
    const long long i = (long long)rank * per + tid;
    const bool live = i < A.N;
    const long long row = b * A.N + (live ? i : 0);

    AlifNeuron nr{};
    if (live) nr = A.nrn[i];
    const df beta{nr.beta_hi, nr.beta_lo}, p{nr.p_hi, nr.p_lo}, c{nr.c_hi, nr.c_lo};
    df v{0.0f, 0.0f}, a{0.0f, 0.0f};
    int rem = 0;
    if (live && A.init) {
        const AlifState s = A.init[row];
        rem = s.rem > 0 ? s.rem : 0;
        v = df{rem > 0 ? 0.0f : s.v, 0.0f};
        a = df{s.a, 0.0f};
    }
    uint32_t word = 0;
    const long long nb = (A.T + TR - 1) / TR;
    // A warp moves its 32 rows' Block chunks (row-contiguous in global memory) with
    // element e = 32 j + lane at row e / cm, step e % cm, so that each access touches a
    // few sectors instead of 32 rows; r and t advance by the quotient and remainder of
    // 32 / cm.
    const long long wrow = (long long)rank * per + warp * 32;  // this warp's first neuron
    const int nrow = (int)(A.N - wrow < 32 ? A.N - wrow : 32);
    const long long grow0 = b * A.N + wrow;
    // feedforward current of Block m into the warp's columns of its accumulator
    auto load_ff = [&](long long m) {
        const long long tb0 = m * TR;
        const int cm = (int)(A.T - tb0 < TR ? A.T - tb0 : TR);
        float *dst = acc + (size_t)(nbuf == 2 ? (int)(m & 1) : 0) * TR * ld + warp * 32;
        const int q32 = 32 / cm, r32 = 32 - q32 * cm;
        int r = lane / cm, t = lane - r * cm;
        for (int e = lane; e < 32 * cm; e += 32) {
            if (r < nrow) cp_async4(dst + (size_t)t * ld + r, A.Iff + (grow0 + r) * A.T + tb0 + t);
            r += q32;
            t += r32;
            if (t >= cm) {
                t -= cm;
                ++r;
            }
        }
    };
    // the Block's FP32 total current (left in cur by the steps) out to I_total, same mapping
    auto store_I = [&](const float *cur, long long tb0, int cm) {
        const int q32 = 32 / cm, r32 = 32 - q32 * cm;
        int r = lane / cm, t = lane - r * cm;
        for (int e = lane; e < 32 * cm; e += 32) {
            if (r < nrow) A.Iout[(grow0 + r) * A.T + tb0 + t] = cur[(size_t)t * ld + warp * 32 + r];
            r += q32;
            t += r32;
            if (t >= cm) {
                t -= cm;
                ++r;
            }
        }
    };
    for (int t = 0; t < TR; ++t) acl[(size_t)t * per + tid] = 0.0f;
    load_ff(0);
    cp_async_commit();
    for (long long n = 0; n < nb; ++n) {
        const long long t0 = n * TR;
        const int cnt = (int)(A.T - t0 < TR ? A.T - t0 : TR);
        // ---- 1. spikes of Block n-1 from every CTA of the cluster, listed as (j, t)
        int total = 0;
        if (n > 0) {
            cl.sync();  // every CTA has published spk[(n-1) & 1]
            const int par = (int)((n - 1) & 1);
            int ts[MAX_G];
            int mine = 0;
#pragma unroll
            for (int r = 0; r < MAX_G; ++r) {
                ts[r] = NO_SPIKE;
                if (r < G && (long long)r * per + tid < A.N) {
                    const int *remote = cl.map_shared_rank(spk + par * per, r);
                    ts[r] = remote[tid];
                }
                mine += ts[r] != NO_SPIKE;
            }
            int incl = mine;
#pragma unroll
            for (int l = 1; l < 32; l <<= 1) {
                const int up = __shfl_up_sync(FULL, incl, l);
                if (lane >= l) incl += up;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const int wv = lane < nwarps ? wsum[lane] : 0;
                int wi = wv;
#pragma unroll
                for (int l = 1; l < 32; l <<= 1) {
                    const int up = __shfl_up_sync(FULL, wi, l);
                    if (lane >= l) wi += up;
                }
                if (lane < nwarps) wsum[lane] = wi - wv;  // exclusive warp offsets
                if (lane == 31) wsum[32] = wi;
            }
            __syncthreads();
            int pos = wsum[warp] + incl - mine;
#pragma unroll
            for (int r = 0; r < MAX_G; ++r)
                if (ts[r] != NO_SPIKE) list[pos++] = ((uint32_t)(r * per + tid) << 10) | (uint32_t)ts[r];
            total = wsum[32];
            __syncthreads();
        }
        // ---- 2. feedforward current plus the recurrent current, column tid of cur.
        // cp.async groups complete in commit order: the weights of the first chunk are
        // committed before the next Block's current, so waiting for all but the newest
        // group leaves only that prefetch in flight.  The loop's trip count is the same
        // in every thread (total is the CTA's), so every lane reaches each __syncwarp.
        float *cur = acc + (size_t)(nbuf == 2 ? (int)(n & 1) : 0) * TR * ld;
        if (nbuf == 1 && n > 0) {
            load_ff(n);
            cp_async_commit();
        }
        {
            const float *Wcol = A.Wt + i;
            bool pref = nbuf == 2 && n + 1 < nb;
            int e0 = 0;
            do {
                const int nch = total - e0 < wch ? total - e0 : wch;
                if (live)
                    for (int k = 0; k < nch; ++k)
                        cp_async4(wbuf + (size_t)k * per + tid, Wcol + (long long)(list[e0 + k] >> 10) * A.N);
                cp_async_commit();
                if (pref) {
                    load_ff(n + 1);
                    cp_async_commit();
                    cp_async_wait<1>();
                    pref = false;
                } else {
                    cp_async_wait<0>();
                }
                __syncwarp();  // the warp's copies of this Block's current are visible to every lane
                if (live)
                    for (int k = 0; k < nch; ++k) {
                        const int t = (int)(list[e0 + k] & 1023u);
                        const df s2 = two_sum(cur[t * ld + tid], wbuf[(size_t)k * per + tid]);
                        cur[t * ld + tid] = s2.hi;
                        acl[t * per + tid] += s2.lo;
                    }
                e0 += nch;
            } while (e0 < total);
        }
        // ---- 3. the Block's steps (state form of Eqs 1-5).  The current of step t + 1 and its
        // product with c do not depend on the state, so they are formed during step t (issue is
        // in order: left inside step t + 1 they would lengthen its dependent chain).
        int sp = NO_SPIKE;
        if (live) {
            // total current of step u in double-single; its FP32 rounding is left in cur for
            // the warp's store below, and acl is cleared for the next Block
            auto take = [&](int u) {
                const df I = quick_two_sum(cur[u * ld + tid], acl[u * per + tid]);
                acl[u * per + tid] = 0.0f;
                cur[u * ld + tid] = I.hi;
                return df_mul(c, I);
            };
            df xn = cnt > 0 ? take(0) : df{0.0f, 0.0f};
            for (int t = 0; t < cnt; ++t) {
                const long long k = t0 + t;
                const df x = xn;
                if (t + 1 < cnt) xn = take(t + 1);
                if (A.ckpt && (k & (ALIF_CKPT_STEPS - 1)) == 0) {
                    AlifState s;
                    s.v = v.hi;
                    s.a = a.hi;
                    s.rem = rem;
                    A.ckpt[row * A.nckpt + k / ALIF_CKPT_STEPS] = s;
                }
                const df V = df_axpy(beta, v, rem == 0 ? x : df{0.0f, 0.0f});  // Eq 2, 4
                // Eq 1 against theta = theta0 + d a (Eq 5).  The FP32 difference dz of V.hi and
                // fl(theta0 + d a.hi) is within 2^-24 (|dz| + |V.hi| + |theta| + |d a.hi|) of the
                // double-single margin, so outside 2^-21 (...) its sign is the margin's; nearer,
                // the threshold is formed in double-single and compared exactly as before.
                const float thf = fmaf(nr.d, a.hi, nr.theta0);
                const float dz = V.hi - thf;
                bool S;
                if (fabsf(dz) > 0x1p-21f * (fabsf(V.hi) + fabsf(thf) + fabsf(nr.d * a.hi))) {
                    S = dz > 0.0f;
                } else {
                    const df th = df_add(df{nr.theta0, 0.0f}, df_mul_f(a, nr.d));
                    S = df_cmp(V, th) > 0;
                }
                if (S) {
                    v = df{0.0f, 0.0f};
                    rem = nr.teff - 1;
                    sp = t;
                } else {
                    v = V;
                    rem = rem > 0 ? rem - 1 : 0;
                }
                a = df_mul(p, a);                       // Eq 5; adding an exact 0 would leave it unchanged
                if (S) a = df_add(a, df{1.0f, 0.0f});
                word |= (S ? 1u : 0u) << (k & 31);
                if ((k & 31) == 31 || k == A.T - 1) {
                    A.spikes[row * A.nwords + (k >> 5)] = word;
                    word = 0;
                }
            }
        }
        if (A.Iout) {
            __syncwarp();
            store_I(cur, t0, cnt);
        }
        spk[(n & 1) * per + tid] = sp;
    }
    if (live && A.fin) {
        AlifState s;
        s.v = v.hi;
        s.a = a.hi;
        s.rem = rem;
        A.fin[row] = s;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Spike raster delayed by D steps: out bit t = in bit t - D (0 for t < D).
__global__ void delay_kernel(long long rows, long long nwords, long long T, long long D, const uint32_t *in,
                             uint32_t *out) {
    const long long total = rows * nwords;
    const long long wsh = D >> 5;
    const int bsh = (int)(D & 31);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / nwords, k = q - r * nwords;
        const long long src = k - wsh;  // word holding bit 32 k - D
        const uint32_t *row = in + r * nwords;
        const uint32_t hi = src >= 0 ? row[src] : 0u;
        const uint32_t lo = (src - 1 >= 0 && bsh) ? row[src - 1] : 0u;
        uint32_t w = bsh ? ((hi << bsh) | (lo >> (32 - bsh))) : hi;
        if (k == nwords - 1 && (T & 31)) w &= (1u << (T & 31)) - 1u;
        out[q] = w;
    }
}

}  // namespace rec

// Returns 0 or a CUDA error code (> 0); -1 when the configuration does not fit.
int launch_alif_forward_recurrent(long long B, long long N, long long T, int TR, const float *Iff, const float *Wt,
                                  const AlifNeuron *nrn, const AlifState *init, float *Iout, uint32_t *spikes,
                                  AlifState *ckpt, AlifState *fin, cudaStream_t stream) {
    using namespace rec;
    Args A;
    A.B = B;
    A.N = N;
    A.T = T;
    A.nwords = (T + 31) / 32;
    A.nckpt = (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS;
    A.TR = TR;
    int G = (int)((N + 127) / 128);
    if (G > MAX_G) G = MAX_G;
    if (G < 1) G = 1;
    int per = (int)((N + G - 1) / G);
    per = (per + 31) & ~31;
    if (per > MAX_PER) return -1;
    A.G = G;
    A.per = per;
    A.Iff = Iff;
    A.Wt = Wt;
    A.nrn = nrn;
    A.init = init;
    A.Iout = Iout;
    A.spikes = spikes;
    A.ckpt = ckpt;
    A.fin = fin;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return (int)e;
    // largest configuration that fits: prefetch first, then as many weights per copy as possible
    size_t smem = 0;
    A.nbuf = 0;
    for (int nbuf = 2; nbuf >= 1 && !A.nbuf; --nbuf)
        for (int wch = MAX_WCH; wch >= 4; wch /= 2) {
            smem = smem_bytes(TR, per, N, nbuf, wch);
            if (smem <= (size_t)optin) {
                A.nbuf = nbuf;
                A.wch = wch;
                break;
            }
        }
    if (!A.nbuf) return -1;
    auto kern = per <= 256 ? rec_fwd_kernel<256> : rec_fwd_kernel<MAX_PER>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B * G), 1, 1);
    cfg.blockDim = dim3((unsigned)per, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, A);
    return (int)e;
}

int launch_delay_spikes(long long rows, long long T, long long D, const uint32_t *in, uint32_t *out,
                        cudaStream_t stream) {
    const long long nwords = (T + 31) / 32;
    const long long total = rows * nwords;
    if (total == 0) return 0;
    long long blocks = (total + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    rec::delay_kernel<<<(unsigned)blocks, 256, 0, stream>>>(rows, nwords, T, D, in, out);
    return (int)cudaGetLastError();
}

}  // namespace alif
