// Event-driven synaptic projection (the feedforward term of Eq 3 / Prop 3):
//     I[b, i, t] = bias_i + sum_{j : S[b, j, t] = 1} W[i, j].
// Input spikes are sparse (a 10-50 Hz input fires at 0.1-0.5 % of 0.1 ms steps),
// so instead of the dense product this visits only the active inputs.
//
// A CTA walks (batch element, 32-step chunk) work units; each thread owns NPT
// consecutive neurons (4 when N allows 16-byte weight rows, so that one load
// and one shared-memory update serve four neurons).  Per unit and block of
// 1024 inputs (1024 / THREADS spike words per thread):
//   1. the CTA builds the chunk's event list in shared memory, grouped by step
//      t and, within a step, in ascending input order (warp bit transposes give
//      the per-(32-input group, step) counts, the groups' counts are scanned per
//      step, every lane writes its own events);
//   2. each thread walks the list in batches of 8 events, loading the 8 weight
//      vectors W_t[j][i .. i+NPT-1] at once (W_t = W transposed: a warp reads
//      32 NPT contiguous floats per event) and adding runs of equal steps in
//      registers into its NPT columns of a [32 steps x 1024 neurons] shared
//      accumulator, started from bias;
// finally each warp writes its 32 NPT neurons' outputs as whole 128-byte row
// segments.  Every sum runs in a fixed order, so the result is deterministic
// and exact up to FP32 rounding (no BF16 split).
#include "common.cuh"

namespace alif {
namespace pev {

constexpr int IN_BLOCK = 1024;      // inputs per event-list pass
constexpr int NB_BLOCK = 1024;      // neurons per pass over the output rows
constexpr int GROUPS = IN_BLOCK / 32;  // 32-input groups per pass
constexpr int MAX_EVENTS = IN_BLOCK * 32;
constexpr int BATCH = 8;            // weights loaded together per thread (one 16-byte list read)
static_assert(IN_BLOCK <= 1024, "an event packs (step << 10) | input within the block");
static_assert(GROUPS == 32, "one scan lane per 32-input group");

template <int NPT>
struct Cfg {
    static constexpr int THREADS = NB_BLOCK / NPT;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int WPT = IN_BLOCK / THREADS;           // spike words per thread and pass
    // floats per step row; with NPT > 1 rows start 16-byte aligned and the columns of row t are
    // permuted (acc_col) so that both the vector updates and the output reads avoid bank conflicts
    static constexpr int ACC_STRIDE = NPT == 1 ? NB_BLOCK + 1 : NB_BLOCK;
    static constexpr size_t ACC_BYTES = ((size_t)32 * ACC_STRIDE * 4 + 15) & ~(size_t)15;
    static constexpr size_t SMEM_BYTES = ACC_BYTES + (size_t)MAX_EVENTS * 2 + GROUPS * 32 * 4 + 33 * 4;
};

template <int NPT>
struct Vec {
    float v[NPT];
};

template <int NPT>
__device__ __forceinline__ Vec<NPT> ldg_vec(const float *p) {
    Vec<NPT> r;
    if constexpr (NPT == 4) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(p));
        r.v[0] = u.x; r.v[1] = u.y; r.v[2] = u.z; r.v[3] = u.w;
    } else if constexpr (NPT == 2) {
        const float2 u = __ldg(reinterpret_cast<const float2 *>(p));
        r.v[0] = u.x; r.v[1] = u.y;
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

template <int NPT>
__device__ __forceinline__ void add_vec(float *p, const float (&x)[NPT]) {
    if constexpr (NPT == 4) {
        float4 *q = reinterpret_cast<float4 *>(p);
        float4 u = *q;
        u.x += x[0]; u.y += x[1]; u.z += x[2]; u.w += x[3];
        *q = u;
    } else if constexpr (NPT == 2) {
        float2 *q = reinterpret_cast<float2 *>(p);
        float2 u = *q;
        u.x += x[0]; u.y += x[1];
        *q = u;
    } else {
        *p += x[0];
    }
}

// Physical column of neuron column `col` in accumulator row t: for NPT > 1 the 4-column groups are
// permuted by bits 2..4 of t (groups stay whole, so vector accesses stay aligned); an output read,
// lane L at rows 4 (L % 8) + i and column 4 q + L / 8, then meets 32 distinct banks.
template <int NPT>
__device__ __forceinline__ int acc_col(int t, int col) {
    return NPT == 1 ? col : (col ^ (((t >> 2) & 7) << 2));
}

struct Args {
    long long B, Nin, N, T, nwords;
    const float *Wt;  // [Nin, N]
    const uint32_t *S;
    const float *bias;
    float *I;
};

template <int NPT>
__global__ void __launch_bounds__(Cfg<NPT>::THREADS, 1) events_kernel(const Args A) {
    using C = Cfg<NPT>;
    constexpr int THREADS = C::THREADS, WARPS = C::WARPS, WPT = C::WPT, ACC_STRIDE = C::ACC_STRIDE;
    extern __shared__ __align__(16) unsigned char smem[];
    float *acc = reinterpret_cast<float *>(smem);                                  // [32][ACC_STRIDE] step x neuron
    uint16_t *list = reinterpret_cast<uint16_t *>(smem + C::ACC_BYTES);            // [MAX_EVENTS] (t << 10) | input
    int *pos = reinterpret_cast<int *>(smem + C::ACC_BYTES + (size_t)MAX_EVENTS * 2);  // [GROUPS][32] first slots
    int *off = pos + GROUPS * 32;                                                  // [33] first event of step t
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long units = A.B * A.nwords;
    const int nblk = (int)((A.Nin + IN_BLOCK - 1) / IN_BLOCK);
    for (long long nb = 0; nb < A.N; nb += NB_BLOCK) {
        const long long i0 = nb + (long long)tid * NPT;  // this thread's first neuron
        float bias[NPT];
        bool live[NPT];
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            live[q] = i0 + q < A.N;
            bias[q] = (A.bias && live[q]) ? A.bias[i0 + q] : 0.0f;
        }
        const bool any_live = live[0];
        for (long long u = blockIdx.x; u < units; u += gridDim.x) {
            const long long b = u / A.nwords, c = u % A.nwords;
            const int nt = (int)(A.T - c * 32 < 32 ? A.T - c * 32 : 32);  // steps in this chunk
#pragma unroll
            for (int t = 0; t < 32; ++t)  // this thread's columns only
#pragma unroll
                for (int q = 0; q < NPT; ++q) acc[t * ACC_STRIDE + acc_col<NPT>(t, tid * NPT) + q] = bias[q];
            for (int blk = 0; blk < nblk; ++blk) {
                // 1a. per-(group, step) event counts: group g of this warp holds inputs
                // g THREADS + 32 warp .. + 31; after the 32x32 bit transpose lane t holds
                // step t's bits of those 32 inputs
                uint32_t tw[WPT];
#pragma unroll
                for (int g = 0; g < WPT; ++g) {
                    const long long j = (long long)blk * IN_BLOCK + g * THREADS + tid;
                    uint32_t w = j < A.Nin ? __ldg(A.S + (b * A.Nin + j) * A.nwords + c) : 0u;
                    if (nt < 32) w &= (1u << nt) - 1u;
                    tw[g] = bits_transpose32(w, lane);
                }
                __syncthreads();  // the previous pass's readers are done with list / pos / off
#pragma unroll
                for (int g = 0; g < WPT; ++g) pos[(g * WARPS + warp) * 32 + lane] = __popc(tw[g]);
                __syncthreads();
                // 1b. step t (t = warp, warp + WARPS, ...): exclusive scan over the 32 groups'
                // counts (lane q = group q) and the step's total; then warp 0 scans the totals
#pragma unroll
                for (int s = 0; s < WPT; ++s) {
                    const int t = warp + s * WARPS;
                    const int n = pos[lane * 32 + t];
                    int incl = n;
#pragma unroll
                    for (int l = 1; l < 32; l <<= 1) {
                        const int up = __shfl_up_sync(FULL, incl, l);
                        if (lane >= l) incl += up;
                    }
                    __syncwarp();
                    pos[lane * 32 + t] = incl - n;  // first slot of (group lane, step t) within step t
                    if (lane == 31) off[t] = incl;  // step t's total, for now
                }
                __syncthreads();
                if (warp == 0) {
                    const int tot = off[lane];
                    int incl = tot;
#pragma unroll
                    for (int l = 1; l < 32; l <<= 1) {
                        const int up = __shfl_up_sync(FULL, incl, l);
                        if (lane >= l) incl += up;
                    }
                    __syncwarp();
                    off[lane] = incl - tot;  // first event of step `lane`
                    if (lane == 31) off[32] = incl;
                }
                __syncthreads();
                // 1c. lane t writes its groups' events of step t, inputs ascending
#pragma unroll
                for (int g = 0; g < WPT; ++g) {
                    const int grp = g * WARPS + warp;
                    int p = off[lane] + pos[grp * 32 + lane];
                    uint32_t m = tw[g];
                    while (m) {
                        const int L = __ffs(m) - 1;
                        m &= m - 1u;
                        list[p++] = (uint16_t)((lane << 10) | (grp * 32 + L));
                    }
                }
                __syncthreads();
                // 2. accumulate this block's events in list order (step, then input)
                if (any_live) {
                    const float *Wb = A.Wt + (long long)blk * IN_BLOCK * A.N + i0;
                    const uint32_t n32 = (uint32_t)A.N;
                    const int col = tid * NPT;
                    const int total = off[32];
                    const int full = total & ~(BATCH - 1);
                    for (int e0 = 0; e0 < full; e0 += BATCH) {
                        const uint4 qv = *reinterpret_cast<const uint4 *>(list + e0);
                        const uint32_t pk[4] = {qv.x, qv.y, qv.z, qv.w};
                        Vec<NPT> wv[BATCH];
                        uint32_t tv[BATCH];
#pragma unroll
                        for (int k = 0; k < BATCH; ++k) {
                            const uint32_t ev = (pk[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                            tv[k] = ev >> 10;
                            wv[k] = ldg_vec<NPT>(Wb + (ev & 1023u) * n32);
                        }
                        // the list is sorted by step: add runs of equal steps in registers and
                        // touch the shared accumulator once per run (the steps are warp-uniform)
                        float run[NPT];
#pragma unroll
                        for (int q = 0; q < NPT; ++q) run[q] = wv[0].v[q];
#pragma unroll
                        for (int k = 1; k < BATCH; ++k) {
                            if (tv[k] == tv[k - 1]) {
#pragma unroll
                                for (int q = 0; q < NPT; ++q) run[q] += wv[k].v[q];
                            } else {
                                add_vec<NPT>(acc + tv[k - 1] * ACC_STRIDE + acc_col<NPT>(tv[k - 1], col), run);
#pragma unroll
                                for (int q = 0; q < NPT; ++q) run[q] = wv[k].v[q];
                            }
                        }
                        add_vec<NPT>(acc + tv[BATCH - 1] * ACC_STRIDE + acc_col<NPT>(tv[BATCH - 1], col), run);
                    }
                    for (int e = full; e < total; ++e) {
                        const uint32_t ev = list[e];
                        const Vec<NPT> w1 = ldg_vec<NPT>(Wb + (ev & 1023u) * n32);
                        const int te = (int)(ev >> 10);
                        add_vec<NPT>(acc + te * ACC_STRIDE + acc_col<NPT>(te, col), w1.v);
                    }
                }
            }
            // 3. the chunk's outputs.  Full chunks: each warp writes its 32 NPT neurons'
            // rows, 4 whole 128-byte row segments per store (lane L: neuron 4 q + L / 8 of
            // the warp, steps 4 (L % 8) .. + 3); the accumulators it reads were written by
            // other threads of the warp, hence the barrier.
            if (nt == 32 && (A.T & 3) == 0 && ((reinterpret_cast<uintptr_t>(A.I) & 15u) == 0)) {
                __syncwarp();
                const int sr = lane >> 3, st = 4 * (lane & 7);
#pragma unroll
                for (int q = 0; q < 8 * NPT; ++q) {
                    const int rr = 4 * q + sr;
                    const long long ii = nb + warp * 32 * NPT + rr;
                    const int cc = warp * 32 * NPT + rr;
                    const float4 v = make_float4(acc[st * ACC_STRIDE + acc_col<NPT>(st, cc)],
                                                 acc[(st + 1) * ACC_STRIDE + acc_col<NPT>(st + 1, cc)],
                                                 acc[(st + 2) * ACC_STRIDE + acc_col<NPT>(st + 2, cc)],
                                                 acc[(st + 3) * ACC_STRIDE + acc_col<NPT>(st + 3, cc)]);
                    if (ii < A.N) *reinterpret_cast<float4 *>(A.I + (b * A.N + ii) * A.T + c * 32 + st) = v;
                }
                __syncwarp();  // the warp's columns are re-initialised by the next unit
            } else {
#pragma unroll
                for (int q = 0; q < NPT; ++q) {
                    if (!live[q]) continue;
                    float *o = A.I + (b * A.N + i0 + q) * A.T + c * 32;
                    for (int t = 0; t < nt; ++t) o[t] = acc[t * ACC_STRIDE + acc_col<NPT>(t, tid * NPT) + q];
                }
            }
        }
    }
}

// W [N, Nin] -> W_t [Nin, N] through 32x32 shared tiles.
__global__ void transpose_kernel(const float *W, long long N, long long Nin, float *Wt) {
    __shared__ float tile[32][33];
    const long long i0 = (long long)blockIdx.y * 32, j0 = (long long)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < N && j < Nin) ? W[i * Nin + j] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long j = j0 + r, i = i0 + threadIdx.x;
        if (j < Nin && i < N) Wt[j * N + i] = tile[threadIdx.x][r];
    }
}

}  // namespace pev

int launch_transpose_weights(const float *W, long long N, long long Nin, float *Wt, cudaStream_t st) {
    if (N == 0 || Nin == 0) return 0;
    const dim3 grid((unsigned)((Nin + 31) / 32), (unsigned)((N + 31) / 32));
    pev::transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(W, N, Nin, Wt);
    return (int)cudaGetLastError();
}

int launch_syn_project_events(long long B, long long Nin, long long N, long long T, const float *Wt,
                              const uint32_t *S, const float *bias, float *I, cudaStream_t st) {
    using namespace pev;
    Args A{B, Nin, N, T, (T + 31) / 32, Wt, S, bias, I};
    const long long units = B * A.nwords;
    if (units == 0 || N == 0) return 0;
    static int sms = 0;
    static bool attr[3] = {false, false, false};
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const unsigned grid = (unsigned)(units < sms ? units : sms);
    // NPT neurons per thread when the weight rows (N floats) and W_t keep NPT-float alignment
    const uintptr_t wa = reinterpret_cast<uintptr_t>(Wt);
    const int npt = (N % 4 == 0 && (wa & 15u) == 0) ? 4 : ((N % 2 == 0 && (wa & 7u) == 0) ? 2 : 1);
    auto go = [&](auto kernel, size_t smem, int threads, int slot) -> int {
        if (!attr[slot]) {
            const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
            attr[slot] = true;
        }
        kernel<<<grid, threads, smem, st>>>(A);
        return (int)cudaGetLastError();
    };
    if (npt == 4) return go(events_kernel<4>, Cfg<4>::SMEM_BYTES, Cfg<4>::THREADS, 2);
    if (npt == 2) return go(events_kernel<2>, Cfg<2>::SMEM_BYTES, Cfg<2>::THREADS, 1);
    return go(events_kernel<1>, Cfg<1>::SMEM_BYTES, Cfg<1>::THREADS, 0);
}

}  // namespace alif
