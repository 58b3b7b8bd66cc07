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
//      transposed, so a warp reads 128 contiguous bytes per spike);
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
constexpr int EB = 8;              // recurrent weights loaded together

struct Args {
    long long B, N, T, nwords, nckpt;
    int TR, G, per;
    const float *Iff;
    const float *Wt;  // [N pre, N post]
    const AlifNeuron *nrn;
    const AlifState *init;
    float *Iout;
    uint32_t *spikes;
    AlifState *ckpt, *fin;
};

__host__ __device__ constexpr size_t smem_bytes(int TR, int per, long long N) {
    return (size_t)2 * TR * per * 4 + (size_t)2 * per * 4 + (size_t)N * 4 + 64 * 4;
}

__global__ void __launch_bounds__(MAX_PER) rec_fwd_kernel(const Args A) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int per = A.per, TR = A.TR, G = A.G;
    float *acc = reinterpret_cast<float *>(smem);                                   // [TR][per] hi
    float *acl = acc + (size_t)TR * per;                                             // [TR][per] lo
    int *spk = reinterpret_cast<int *>(smem + (size_t)2 * TR * per * 4);             // [2][per]
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
    const float *Irow = A.Iff + row * A.T;
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
        // ---- 2. feedforward current plus the recurrent current, column tid of acc
        if (live) {
            for (int tb = 0; tb < cnt; tb += EB) {  // EB loads in flight, then their stores
                float x[EB];
#pragma unroll
                for (int k = 0; k < EB; ++k) x[k] = tb + k < cnt ? __ldg(Irow + t0 + tb + k) : 0.0f;
#pragma unroll
                for (int k = 0; k < EB; ++k)
                    if (tb + k < cnt) {
                        acc[(tb + k) * per + tid] = x[k];
                        acl[(tb + k) * per + tid] = 0.0f;
                    }
            }
            const float *Wcol = A.Wt + i;
            // EB weights in flight at a time: the loads are independent, the adds are not
            int e = 0;
            for (; e + EB <= total; e += EB) {
                uint32_t ev[EB];
                float wv[EB];
#pragma unroll
                for (int k = 0; k < EB; ++k) {
                    ev[k] = list[e + k];
                    wv[k] = __ldg(Wcol + (long long)(ev[k] >> 10) * A.N);
                }
#pragma unroll
                for (int k = 0; k < EB; ++k) {
                    const int q = (int)(ev[k] & 1023u) * per + tid;
                    const df s2 = two_sum(acc[q], wv[k]);
                    acc[q] = s2.hi;
                    acl[q] += s2.lo;
                }
            }
            for (; e < total; ++e) {
                const uint32_t ev = list[e];
                const int q = (int)(ev & 1023u) * per + tid;
                const df s2 = two_sum(acc[q], __ldg(Wcol + (long long)(ev >> 10) * A.N));
                acc[q] = s2.hi;
                acl[q] += s2.lo;
            }
        }
        // ---- 3. the Block's steps (state form of Eqs 1-5)
        int sp = NO_SPIKE;
        if (live) {
            for (int t = 0; t < cnt; ++t) {
                const long long k = t0 + t;
                if (A.ckpt && (k & (ALIF_CKPT_STEPS - 1)) == 0) {
                    AlifState s;
                    s.v = v.hi;
                    s.a = a.hi;
                    s.rem = rem;
                    A.ckpt[row * A.nckpt + k / ALIF_CKPT_STEPS] = s;
                }
                const df I = quick_two_sum(acc[t * per + tid], acl[t * per + tid]);
                if (A.Iout) A.Iout[row * A.T + k] = I.hi;
                const df V = df_add(df_mul(beta, v), rem == 0 ? df_mul(c, I) : df{0.0f, 0.0f});  // Eq 2, 4
                const df th = df_add(df{nr.theta0, 0.0f}, df_mul_f(a, nr.d));                      // Eq 5
                const bool S = df_cmp(V, th) > 0;                                                 // Eq 1
                if (S) {
                    v = df{0.0f, 0.0f};
                    rem = nr.teff - 1;
                    sp = t;
                } else {
                    v = V;
                    rem = rem > 0 ? rem - 1 : 0;
                }
                a = df_add(df_mul(p, a), df{S ? 1.0f : 0.0f, 0.0f});
                word |= (S ? 1u : 0u) << (k & 31);
                if ((k & 31) == 31 || k == A.T - 1) {
                    A.spikes[row * A.nwords + (k >> 5)] = word;
                    word = 0;
                }
            }
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

size_t recurrent_smem_bytes(int TR, int per, long long N) { return rec::smem_bytes(TR, per, N); }

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
    const size_t smem = smem_bytes(TR, per, N);
    if (smem > 200 * 1024) return -1;
    cudaError_t e = cudaFuncSetAttribute(rec_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    e = cudaLaunchKernelEx(&cfg, rec_fwd_kernel, A);
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
