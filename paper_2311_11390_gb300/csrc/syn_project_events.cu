// Event-driven synaptic projection (the feedforward term of Eq 3 / Prop 3):
//     I[b, i, t] = bias_i + sum_{j : S[b, j, t] = 1} W[i, j].
// Input spikes are sparse (a 10-50 Hz input fires at 0.1-0.5 % of 0.1 ms steps),
// so instead of the dense product this visits only the active inputs.
//
// A CTA of 1024 threads walks (batch element, 32-step chunk) work units.  Per
// unit and block of 1024 inputs (one spike word per thread):
//   1. the CTA builds the chunk's event list in shared memory, grouped by step
//      t and, within a step, in ascending input order (warp ballots give the
//      per-(warp, step) counts, one warp scans them into positions, every
//      thread writes its own events);
//   2. each thread (one neuron) walks the list in batches of 8 events, loading
//      the 8 weights W_t[j][i] at once (W_t = W transposed, so a warp reads 128
//      contiguous bytes per event) and adding each into its accumulator for
//      the event's step: a column of a [32 steps x 1024 threads] shared array,
//      started from bias_i;
// (runs of equal steps within a batch are summed in registers first, so the
// shared accumulator is read and written once per run); finally each warp
// writes its 32 neurons' outputs as whole 128-byte row segments.  Every sum runs in a fixed order, so the
// result is deterministic and exact up to FP32 rounding (no BF16 split).
#include "common.cuh"

namespace alif {
namespace pev {

constexpr int THREADS = 1024;
constexpr int WARPS = THREADS / 32;
constexpr int IN_BLOCK = THREADS;  // inputs per event-list pass (one word per thread)
constexpr int MAX_EVENTS = IN_BLOCK * 32;
constexpr int BATCH = 8;            // weights loaded together per thread (one 16-byte list read)
constexpr int ACC_STRIDE = THREADS + 1;  // floats per step row: (t, i) and (t', i) in different banks
constexpr size_t ACC_BYTES = ((size_t)32 * ACC_STRIDE * 4 + 15) & ~(size_t)15;
constexpr size_t SMEM_BYTES = ACC_BYTES + (size_t)MAX_EVENTS * 2 + WARPS * 32 * 4 + 33 * 4;
static_assert(IN_BLOCK <= 1024, "an event packs (step << 10) | input within the block");
static_assert(WARPS == 32, "warp t scans the counts of step t");

struct Args {
    long long B, Nin, N, T, nwords;
    const float *Wt;  // [Nin, N]
    const uint32_t *S;
    const float *bias;
    float *I;
};

__global__ void __launch_bounds__(THREADS, 1) events_kernel(const Args A) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *acc = reinterpret_cast<float *>(smem);                              // [32][ACC_STRIDE] step x neuron
    uint16_t *list = reinterpret_cast<uint16_t *>(smem + ACC_BYTES);           // [MAX_EVENTS] (t << 10) | input
    int *pos = reinterpret_cast<int *>(smem + ACC_BYTES + (size_t)MAX_EVENTS * 2);  // [WARPS][32] first slots
    int *off = pos + WARPS * 32;                                               // [33] first event of step t
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long units = A.B * A.nwords;
    const int nblk = (int)((A.Nin + IN_BLOCK - 1) / IN_BLOCK);
    for (long long nb = 0; nb < A.N; nb += THREADS) {
        const long long i = nb + tid;
        const bool live = i < A.N;
        const float bias = (A.bias && live) ? A.bias[i] : 0.0f;
        for (long long u = blockIdx.x; u < units; u += gridDim.x) {
            const long long b = u / A.nwords, c = u % A.nwords;
            const int nt = (int)(A.T - c * 32 < 32 ? A.T - c * 32 : 32);  // steps in this chunk
#pragma unroll
            for (int t = 0; t < 32; ++t) acc[t * ACC_STRIDE + tid] = bias;  // this thread's column only
            for (int blk = 0; blk < nblk; ++blk) {
                const long long j = (long long)blk * IN_BLOCK + tid;
                uint32_t w = j < A.Nin ? __ldg(A.S + (b * A.Nin + j) * A.nwords + c) : 0u;
                if (nt < 32) w &= (1u << nt) - 1u;
                // 1a. per-(warp, step) event counts: after the 32x32 bit transpose lane t
                // holds step t's bits of the warp's 32 inputs
                const uint32_t tw = bits_transpose32(w, lane);
                const int mine = __popc(tw);
                __syncthreads();  // the previous pass's readers are done with list / pos / off
                pos[warp * 32 + lane] = mine;
                __syncthreads();
                // 1b. warp t: exclusive scan over the 32 warps' counts of step t (lane q =
                // warp q) and the step's total; then warp 0 scans the totals over steps
                {
                    const int t = warp;
                    const int n = pos[lane * 32 + t];
                    int incl = n;
#pragma unroll
                    for (int l = 1; l < 32; l <<= 1) {
                        const int up = __shfl_up_sync(FULL, incl, l);
                        if (lane >= l) incl += up;
                    }
                    __syncthreads();  // every count is read before it is overwritten
                    pos[lane * 32 + t] = incl - n;  // first slot of (warp lane, step t) within step t
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
                // 1c. lane t writes the warp's events of step t, inputs ascending
                {
                    int p = off[lane] + pos[warp * 32 + lane];
                    uint32_t m = tw;
                    while (m) {
                        const int L = __ffs(m) - 1;
                        m &= m - 1u;
                        list[p++] = (uint16_t)((lane << 10) | (warp * 32 + L));
                    }
                }
                __syncthreads();
                // 2. accumulate this block's events in list order (step, then input):
                // 8 list entries per 16-byte shared load, their 8 weights loaded together
                if (live) {
                    const float *Wb = A.Wt + (long long)blk * IN_BLOCK * A.N + i;
                    const uint32_t n32 = (uint32_t)A.N;
                    float *accp = acc + tid;
                    const int total = off[32];
                    const int full = total & ~(BATCH - 1);
                    for (int e0 = 0; e0 < full; e0 += BATCH) {
                        const uint4 q = *reinterpret_cast<const uint4 *>(list + e0);
                        const uint32_t pk[4] = {q.x, q.y, q.z, q.w};
                        float wv[BATCH];
                        uint32_t tv[BATCH];
#pragma unroll
                        for (int k = 0; k < BATCH; ++k) {
                            const uint32_t ev = (pk[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                            tv[k] = ev >> 10;
                            wv[k] = __ldg(Wb + (ev & 1023u) * n32);
                        }
                        // the list is sorted by step: add runs of equal steps in registers and
                        // touch the shared accumulator once per run (the steps are warp-uniform)
                        float run = wv[0];
#pragma unroll
                        for (int k = 1; k < BATCH; ++k) {
                            if (tv[k] == tv[k - 1]) {
                                run += wv[k];
                            } else {
                                accp[tv[k - 1] * ACC_STRIDE] += run;
                                run = wv[k];
                            }
                        }
                        accp[tv[BATCH - 1] * ACC_STRIDE] += run;
                    }
                    for (int e = full; e < total; ++e) {
                        const uint32_t ev = list[e];
                        accp[(ev >> 10) * ACC_STRIDE] += __ldg(Wb + (ev & 1023u) * n32);
                    }
                }
            }
            // 3. the chunk's outputs.  Full chunks: each warp writes its 32 neurons' rows,
            // 4 whole 128-byte row segments per store (lane L: neuron 4 q + L / 8 of the
            // warp, steps 4 (L % 8) .. + 3); the accumulators it reads were written by
            // other threads of the warp, hence the barrier.
            if (nt == 32 && (A.T & 3) == 0 && ((reinterpret_cast<uintptr_t>(A.I) & 15u) == 0)) {
                __syncwarp();
                const int sr = lane >> 3, st = 4 * (lane & 7);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int rr = 4 * q + sr;
                    const long long ii = nb + warp * 32 + rr;
                    const float *ap = acc + st * ACC_STRIDE + warp * 32 + rr;
                    const float4 v = make_float4(ap[0], ap[ACC_STRIDE], ap[2 * ACC_STRIDE], ap[3 * ACC_STRIDE]);
                    if (ii < A.N) *reinterpret_cast<float4 *>(A.I + (b * A.N + ii) * A.T + c * 32 + st) = v;
                }
                __syncwarp();  // the warp's columns are re-initialised by the next unit
            } else if (live) {
                float *o = A.I + (b * A.N + i) * A.T + c * 32;
#pragma unroll
                for (int t = 0; t < 32; ++t)
                    if (t < nt) o[t] = acc[t * ACC_STRIDE + tid];
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
    static bool attr = false;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(events_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return (int)e;
        attr = true;
    }
    const unsigned grid = (unsigned)(units < sms ? units : sms);
    events_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(A);
    return (int)cudaGetLastError();
}

}  // namespace alif
