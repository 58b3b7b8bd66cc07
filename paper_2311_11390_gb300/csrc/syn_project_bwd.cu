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
// g_S is a dense FP32 GEMM (W^T x g_I per batch element) on the CUDA cores.
#include "common.cuh"

namespace alif {
namespace pbwd {

constexpr int TI = 32;       // neuron rows per CTA (one per lane)
constexpr int JT = 1024;     // inputs per CTA (shared-memory accumulator columns)
constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;

// partial[b][i][j] (j < ldp) and partial_bias[b][i]; blockIdx.z selects inputs [z*JT, z*JT+JT).
// Time runs in super-chunks of SC spike words (SC * 32 steps): the CTA stages g_I of its 32 rows
// for the whole super-chunk, then each lane (one input) reads its SC consecutive words -- 4 SC
// contiguous bytes, so after the first the loads hit L1 -- and the warp visits only the inputs
// whose word is nonzero (ballot), adding the staged g_I of every set bit.
constexpr int SC = 8;
constexpr int GT_STRIDE = SC * 32 + 1;  // staged row stride (floats): lanes hit distinct banks
__global__ void __launch_bounds__(THREADS) gw_events_kernel(const float *__restrict__ gI,
                                                            const uint32_t *__restrict__ S, long long B,
                                                            long long N, long long Nin, long long T, int nwin,
                                                            int ldp, float *part, float *part_b) {
    extern __shared__ float sm[];
    const long long jbase = (long long)blockIdx.z * JT;
    const int jn = (int)(Nin - jbase < JT ? Nin - jbase : JT);  // inputs of this CTA
    const int jcap = (int)(Nin < JT ? Nin : JT);  // accumulator columns allocated (same for every CTA)
    float *acc = sm;                      // [jcap][TI] (column j, lane i) -> conflict-free
    float *gt = sm + (size_t)jcap * TI;   // [TI][GT_STRIDE] staged g_I (row i, step t)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long b = blockIdx.y;
    const long long i0 = (long long)blockIdx.x * TI;
    for (int k = tid; k < jn * TI; k += THREADS) acc[k] = 0.0f;
    float bias_acc = 0.0f;
    const long long row = i0 + lane;
    for (int tw0 = 0; tw0 < nwin; tw0 += SC) {
        const long long tb = (long long)tw0 * 32;
        __syncthreads();  // previous super-chunk consumed
        // stage g_I[b, i0..i0+31, tb .. tb + 32 SC): warp w loads rows w, w+8, ... coalesced along t
        for (int r = warp; r < TI; r += WARPS) {
            const long long gi = i0 + r;
            const float *src = gI + (b * N + (gi < N ? gi : 0)) * T + tb;
#pragma unroll
            for (int c = lane; c < SC * 32; c += 32)
                gt[r * GT_STRIDE + c] = (gi < N && tb + c < T) ? src[c] : 0.0f;
        }
        __syncthreads();
        if (warp == 0 && blockIdx.z == 0) {
#pragma unroll 8
            for (int c = 0; c < SC * 32; ++c) bias_acc += gt[lane * GT_STRIDE + c];
        }
        // events: warp w handles input groups j0 = 32 w, 32 (w + 8), ...; lanes are neuron rows
        for (int j0 = warp * 32; j0 < jn; j0 += WARPS * 32) {
            const int jl = j0 + lane;
            const uint32_t *srow = S + (b * Nin + jbase + (jl < jn ? jl : 0)) * nwin;
            uint32_t wv[SC];
#pragma unroll
            for (int q = 0; q < SC; ++q) {
                const int tw = tw0 + q;
                wv[q] = (jl < jn && tw < nwin) ? __ldg(srow + tw) : 0u;
                if (tw == nwin - 1 && (T & 31)) wv[q] &= (1u << (T & 31)) - 1u;
            }
#pragma unroll
            for (int q = 0; q < SC; ++q) {
                uint32_t nz = __ballot_sync(FULL, wv[q] != 0u);
                while (nz) {  // warp-uniform: the inputs of this group with a spike in word q
                    const int L = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    uint32_t wq = __shfl_sync(FULL, wv[q], L);
                    float sum = 0.0f;
                    while (wq) {
                        const int t = __ffs(wq) - 1;
                        wq &= wq - 1u;
                        sum += gt[lane * GT_STRIDE + q * 32 + t];
                    }
                    acc[(size_t)(j0 + L) * TI + lane] += sum;
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
    if (warp == 0 && blockIdx.z == 0 && row < N) part_b[b * N + row] = bias_acc;
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

// g_S[b, j, t] = sum_i W[i, j] g_I[b, i, t]: tiled FP32 GEMM, 64 (j) x 128 (t) per CTA,
// K = neurons in steps of 16, 256 threads with 8 x 4 outputs each.
constexpr int GJ = 64, GT = 128, GK = 16;
__global__ void __launch_bounds__(256) gs_gemm_kernel(const float *__restrict__ W, const float *__restrict__ gI,
                                                     long long N, long long Nin, long long T, float *gS) {
    __shared__ float Ws[GK][GJ + 4];   // W[i, j] tile (k = i)
    __shared__ float Gs[GK][GT + 4];   // gI[b, i, t] tile
    const int tid = threadIdx.x;
    const long long b = blockIdx.z;
    const long long j0 = (long long)blockIdx.y * GJ, t0 = (long long)blockIdx.x * GT;
    const int tj = (tid / 32) * 8;     // 8 warps x 8 rows of j
    const int tt = (tid % 32) * 4;     // 32 lanes x 4 steps
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
    for (long long k0 = 0; k0 < N; k0 += GK) {
        // load W tile: 16 x 64 = 1024 values, 4 per thread (coalesced along j)
        for (int e = tid; e < GK * GJ; e += 256) {
            const int kk = e / GJ, jj = e % GJ;
            const long long i = k0 + kk, j = j0 + jj;
            Ws[kk][jj] = (i < N && j < Nin) ? W[i * Nin + j] : 0.0f;
        }
        // load g_I tile: 16 x 128 = 2048 values, 8 per thread (coalesced along t)
        for (int e = tid; e < GK * GT; e += 256) {
            const int kk = e / GT, ttt = e % GT;
            const long long i = k0 + kk, t = t0 + ttt;
            Gs[kk][ttt] = (i < N && t < T) ? gI[(b * N + i) * T + t] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float wv[8], gv[4];
#pragma unroll
            for (int r = 0; r < 8; ++r) wv[r] = Ws[kk][tj + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) gv[c] = Gs[kk][tt + c];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(wv[r], gv[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const long long j = j0 + tj + r;
        if (j >= Nin) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long t = t0 + tt + c;
            if (t < T) gS[(b * Nin + j) * T + t] = acc[r][c];
        }
    }
}

}  // namespace pbwd

size_t syn_project_backward_ws(long long B, long long N, long long Nin) {
    const long long ldp = (Nin + 3) & ~3LL;
    return (size_t)(B * N * ldp + B * N) * sizeof(float);
}

int launch_syn_project_backward(long long B, long long Nin, long long N, long long T, const float *W,
                                const uint32_t *S, const float *gI, float *gW, float *gS, float *gb, void *ws,
                                cudaStream_t stream) {
    using namespace pbwd;
    if ((gW || gb) && Nin > 0) {
        const int ldp = (int)((Nin + 3) & ~3LL);
        float *part = static_cast<float *>(ws);
        float *part_b = part + B * N * ldp;
        const long long jt = Nin < JT ? Nin : JT;
        const size_t smem = ((size_t)jt * TI + (size_t)TI * GT_STRIDE) * sizeof(float);
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
        const dim3 grid((unsigned)((T + GT - 1) / GT), (unsigned)((Nin + GJ - 1) / GJ), (unsigned)B);
        gs_gemm_kernel<<<grid, 256, 0, stream>>>(W, gI, N, Nin, T, gS);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}

}  // namespace alif
