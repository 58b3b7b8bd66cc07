// Backward of the synaptic projection (Eq 3 / Prop 3 feedforward term):
//   g_W[i, j]   = sum_{b,t} g_I[b, i, t] S[b, j, t]
//   g_bias[i]   = sum_{b,t} g_I[b, i, t]
//   g_S[b, j, t] = sum_i W[i, j] g_I[b, i, t]
// g_W and g_bias are event-driven: input spikes are sparse, so for every
// (batch element, 32-row neuron tile) a CTA stages g_I 256 steps at a time in
// shared memory and its warps walk the set bits of the inputs' spike words;
// at each spike every lane (one neuron row) adds its staged g_I value to its
// accumulator column in shared memory.  Per-(b, row) partials go to a
// workspace and are summed over the batch in a fixed order (deterministic).
// g_S is a dense product (W^T x g_I per batch element) on the tcgen05 tensor cores with both
// operands split into two BF16 terms (syn_grad_input.cu).
#include "common.cuh"

namespace alif {
namespace pbwd {

constexpr int TI = 32;       // neuron rows per CTA (one per lane)
constexpr int JT = 1024;     // inputs per CTA (shared-memory accumulator columns)
constexpr int WARPS = 32;    // one warp per 32-input group and per staged row
constexpr int THREADS = WARPS * 32;

// partial[b][i][j] (j < ldp) and partial_bias[b][i]; blockIdx.z selects inputs [z*JT, z*JT+JT).
// Time runs in super-chunks of SC spike words (SC * 32 steps).  The CTA stages g_I of its 32 rows
// for a super-chunk into one of two buffers (cp.async, one super-chunk ahead, warp w copying row w
// coalesced along t), so the next super-chunk's load overlaps this one's events.  Warp w handles
// input group w: load k of lane l reads word (l % 8) of input 4 k + l / 8, so that eight lanes read
// one input's SC = 8 consecutive words (32 bytes) and a load touches four sectors (the next
// super-chunk's words are read ahead).  The warp visits only the nonzero words (ballot over each
// load, lanes in order: for one input its words in time order), every lane (one neuron row) adding
// the staged g_I of each set bit.  A thread's bias partial covers the steps c = lane + 32 k of row
// `warp`; the warp's lanes are summed in a fixed shuffle order at the end.
constexpr int SC = 8;
constexpr int GT_STRIDE = SC * 32 + 1;  // staged row stride (floats): lanes hit distinct banks

__device__ __forceinline__ void cp_async4_zfill(float *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}

__global__ void __launch_bounds__(THREADS) gw_events_kernel(const float *__restrict__ gI,
                                                            const uint32_t *__restrict__ S, long long B,
                                                            long long N, long long Nin, long long T, int nwin,
                                                            int ldp, float *part, float *part_b) {
    extern __shared__ float sm[];
    const long long jbase = (long long)blockIdx.z * JT;
    const int jn = (int)(Nin - jbase < JT ? Nin - jbase : JT);  // inputs of this CTA
    const int jcap = (int)(Nin < JT ? Nin : JT);  // accumulator columns allocated (same for every CTA)
    float *acc = sm;                      // [jcap][TI] (column j, lane i) -> conflict-free
    float *gt = sm + (size_t)jcap * TI;   // [2][TI][GT_STRIDE] staged g_I (row i, step t)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long b = blockIdx.y;
    const long long i0 = (long long)blockIdx.x * TI;
    for (int k = tid; k < jn * TI; k += THREADS) acc[k] = 0.0f;
    const int nsc = (nwin + SC - 1) / SC;
    // row `warp` of the tile, steps tb + lane + 32 k, into buffer buf (zeros past N or T)
    const long long srow_g = i0 + warp;
    const float *grow = gI + (b * N + (srow_g < N ? srow_g : 0)) * T;
    auto stage = [&](int sc, int buf) {
        const long long tb = (long long)sc * SC * 32;
        float *dst = gt + ((size_t)buf * TI + warp) * GT_STRIDE;
#pragma unroll
        for (int k = 0; k < SC; ++k) {
            const long long t = tb + lane + 32 * k;
            const bool ok = srow_g < N && t < T;
            cp_async4_zfill(dst + lane + 32 * k, ok ? grow + t : grow, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // the group's spike words: load k of this lane is word q = lane % 8 of input 4 k + lane / 8
    static_assert(SC == 8, "eight lanes per input");
    const int j0 = warp * 32;
    const int lq = lane & 7, lj = lane >> 3;
    const uint32_t tail = (T & 31) ? (1u << (T & 31)) - 1u : ~0u;  // valid bits of the last word
    // word q = lq of input j0 + 4 k + lj at super-chunk sc: wp + 4 k nwin + SC sc
    const uint32_t *wp = S + (b * Nin + jbase + (j0 + lj < jn ? j0 + lj : 0)) * nwin + lq;
    const long long kstride = 4LL * nwin;
    unsigned kvalid = 0;  // bit k: input j0 + 4 k + lj exists
#pragma unroll
    for (int k = 0; k < SC; ++k) kvalid |= (j0 + 4 * k + lj < jn ? 1u : 0u) << k;
    auto word = [&](int k, int sc) -> uint32_t {
        const int tw = sc * SC + lq;
        if (!((kvalid >> k) & 1u) || tw >= nwin) return 0u;
        const uint32_t v = __ldg(wp + k * kstride + sc * SC);
        return tw == nwin - 1 ? v & tail : v;
    };
    float bias_acc = 0.0f;
    uint32_t wn[SC];
#pragma unroll
    for (int k = 0; k < SC; ++k) wn[k] = word(k, 0);
    stage(0, 0);
    for (int sc = 0; sc < nsc; ++sc) {
        const int buf = sc & 1;
        __syncthreads();  // every warp is done with the other buffer (super-chunk sc - 1)
        if (sc + 1 < nsc) {
            stage(sc + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();  // super-chunk sc staged by every thread's copies
        const float *g = gt + (size_t)buf * TI * GT_STRIDE;
        const float *gl = g + lane * GT_STRIDE;  // this lane's (neuron row's) staged g_I
        if (blockIdx.z == 0) {
#pragma unroll
            for (int k = 0; k < SC; ++k) bias_acc += g[warp * GT_STRIDE + lane + 32 * k];
        }
        uint32_t wv[SC];
#pragma unroll
        for (int k = 0; k < SC; ++k) {
            wv[k] = wn[k];
            wn[k] = sc + 1 < nsc ? word(k, sc + 1) : 0u;  // next super-chunk's words, read ahead
        }
        if (j0 < jn) {
#pragma unroll
            for (int k = 0; k < SC; ++k) {
                uint32_t nz = __ballot_sync(FULL, wv[k] != 0u);
                float *ak = acc + (size_t)(j0 + 4 * k) * TI + lane;
                while (nz) {  // warp-uniform: the nonzero words of inputs 4 k .. 4 k + 3
                    const int L = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    uint32_t wq = __shfl_sync(FULL, wv[k], L);
                    const float *gq = gl + (L & 7) * 32;
                    float sum = gq[__ffs(wq) - 1];  // most words hold one spike
                    wq &= wq - 1u;
                    while (wq) {
                        const int t = __ffs(wq) - 1;
                        wq &= wq - 1u;
                        sum += gq[t];
                    }
                    ak[(L >> 3) * TI] += sum;
                }
            }
        }
    }
    __syncthreads();
    // write this (b, row-tile, input-tile)'s partial: part[b][i][jbase + j]
    for (int k = tid; k < jn * TI; k += THREADS) {
        const int j = k / TI, r = k % TI;
        const long long gi = i0 + r;
        if (gi < N) part[(b * N + gi) * ldp + jbase + j] = acc[k];
    }
    if (blockIdx.z == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bias_acc += __shfl_xor_sync(FULL, bias_acc, o);
        if (lane == 0 && srow_g < N) part_b[b * N + srow_g] = bias_acc;
    }
}

// Fixed-order sum over the batch: g_W[i][j] = sum_b part[b][i][j]; g_bias[i] likewise.
__global__ void gw_reduce_kernel(const float *part, const float *part_b, long long B, long long N, long long Nin,
                                 int ldp, float *gW, float *gb) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N * Nin) {
        const long long i = k / Nin, j = k % Nin;
        float s = 0.0f;
        for (long long b = 0; b < B; ++b) s += part[(b * N + i) * ldp + j];
        if (gW) gW[k] = s;
    }
    if (gb && k < N) {
        float s = 0.0f;
        for (long long b = 0; b < B; ++b) s += part_b[b * N + k];
        gb[k] = s;
    }
}

}  // namespace pbwd

size_t syn_grad_input_ws(long long N, long long Nin);
int launch_syn_grad_input(long long B, long long N, long long Nin, long long T, const float *W, const float *gI,
                          float *gS, void *ws, int *status, cudaStream_t stream);

// Workspace: the per-batch-element partials of g_W and g_bias, then (256-byte aligned) the BF16
// terms of W^T for g_S.
static size_t gw_part_bytes(long long B, long long N, long long Nin) {
    const long long ldp = (Nin + 3) & ~3LL;
    return ((size_t)(B * N * ldp + B * N) * sizeof(float) + 255) & ~(size_t)255;
}

size_t syn_project_backward_ws(long long B, long long N, long long Nin) {
    return gw_part_bytes(B, N, Nin) + syn_grad_input_ws(N, Nin);
}

int launch_syn_project_backward(long long B, long long Nin, long long N, long long T, const float *W,
                                const uint32_t *S, const float *gI, float *gW, float *gS, float *gb, void *ws,
                                int *status, cudaStream_t stream) {
    using namespace pbwd;
    if ((gW || gb) && Nin > 0) {
        const int ldp = (int)((Nin + 3) & ~3LL);
        float *part = static_cast<float *>(ws);
        float *part_b = part + B * N * ldp;
        const long long jt = Nin < JT ? Nin : JT;
        const size_t smem = ((size_t)jt * TI + (size_t)2 * TI * GT_STRIDE) * sizeof(float);
        static size_t attr = 0;
        if (smem > attr) {
            if (cudaFuncSetAttribute(gw_events_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return (int)cudaGetLastError();
            attr = smem;
        }
        const dim3 grid((unsigned)((N + TI - 1) / TI), (unsigned)B, (unsigned)((Nin + JT - 1) / JT));
        gw_events_kernel<<<grid, THREADS, smem, stream>>>(gI, S, B, N, Nin, T, (int)((T + 31) / 32), ldp, part,
                                                          part_b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
        const long long total = N * Nin > N ? N * Nin : N;
        gw_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(part, part_b, B, N, Nin, ldp, gW, gb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    if (gS) {
        void *gws = static_cast<unsigned char *>(ws) + gw_part_bytes(B, N, Nin);
        const int rc = launch_syn_grad_input(B, N, Nin, T, W, gI, gS, gws, status, stream);
        if (rc) return rc;
    }
    return 0;
}

}  // namespace alif
