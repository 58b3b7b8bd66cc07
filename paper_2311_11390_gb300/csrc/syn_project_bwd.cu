// Backward of the synaptic projection (Eq 3 / Prop 3 feedforward term):
//   g_W[i, j]   = sum_{b,t} g_I[b, i, t] S[b, j, t]
//   g_bias[i]   = sum_{b,t} g_I[b, i, t]
//   g_S[b, j, t] = sum_i W[i, j] g_I[b, i, t]
// g_W and g_bias are event-driven: input spikes are sparse, so for every
// (batch element, 16-row neuron tile) a CTA stages g_I 512 steps at a time in
// shared memory and each thread, owning one input, walks that input's spikes,
// adding the staged g_I column of the 16 rows to its accumulators.  Per-(b, row)
// partials go to a workspace and are summed over the batch in a fixed order
// (deterministic).
// g_S is a dense product (W^T x g_I per batch element) on the tcgen05 tensor cores with both
// operands split into two BF16 terms (syn_grad_input.cu).
#include "common.cuh"

namespace alif {
namespace pbwd {

// g_W and g_bias with one thread per input.  A CTA covers (batch element b, 16 neuron rows,
// up to 1024 inputs); thread j accumulates g_W[i0 .. i0+15][j] in registers.  Time runs in
// 512-step chunks: the CTA stages g_I of its 16 rows step-major (gt[t][row], 80-byte step rows,
// the next chunk's values prefetched into registers while this chunk's events are processed).
// Each thread's 16 spike words of a chunk arrive by cp.async in its own shared-memory slot
// (double-buffered, one chunk ahead); the thread takes the mask of the nonzero ones and walks its
// spikes in step order, one per iteration across the warp (the next nonzero word fetched from the
// slot when the current one is exhausted), adding the staged column g_I[i0 .. i0+15][t] with four
// 16-byte reads.  Every sum runs in step order: deterministic.
constexpr int LR = 16;          // neuron rows per CTA (accumulators per thread)
constexpr int LJ = 1024;        // inputs per CTA, one per thread
constexpr int LTHREADS = LJ;
constexpr int LCH = 512;        // steps per chunk
constexpr int LCW = LCH / 32;   // spike words per input and chunk
constexpr int LGS = LR + 4;     // floats per staged step row (80 bytes: 16-byte aligned)
constexpr size_t LSMEM = (size_t)LCH * LGS * 4 + (size_t)2 * LCW * LTHREADS * 4 + 64 * LR * 4;

__device__ __forceinline__ void cp_async16_zfill(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// 16-byte unit of word group m (words 4m .. 4m+3) in thread tid's 64-byte slot, swizzled so that a
// quarter warp's 16-byte accesses to the same group fall in distinct bank groups
__device__ __forceinline__ int slot_unit(int tid, int m) { return 4 * tid + (m ^ ((tid >> 1) & 3)); }

template <bool VG, bool VS>  // VG: g_I rows in 16-byte units (T % 4 == 0); VS: spike words in 16-byte units
__global__ void __launch_bounds__(LTHREADS, 1) gw_lane_kernel(const float *__restrict__ gI,
                                                              const uint32_t *__restrict__ S, long long N,
                                                              long long Nin, long long T, int nwin, int ldp,
                                                              float *part, float *part_b) {
    extern __shared__ float sm[];
    float *gt = sm;                                                          // [LCH][LGS]
    uint32_t *wsl = reinterpret_cast<uint32_t *>(sm + (size_t)LCH * LGS);   // [2][LTHREADS][LCW] word slots
    float *bsm = sm + (size_t)LCH * LGS + (size_t)2 * LCW * LTHREADS;       // [64][LR]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long b = blockIdx.y;
    const long long i0 = (long long)blockIdx.x * LR;
    const long long j = (long long)blockIdx.z * LJ + tid;
    const bool jv = j < Nin;
    const int nch = (int)((T + LCH - 1) / LCH);
    const uint32_t tail = (T & 31) ? (1u << (T & 31)) - 1u : ~0u;  // valid bits of the last word
    const uint32_t *wrow = S + (b * Nin + (jv ? j : 0)) * (long long)nwin;
    // staging map: row r = lane & 15, 16-byte units q = 4 warp + 2 h + lane / 16 (h = 0, 1): a
    // half warp reads 16 rows at one step group, and its stores to gt[t][r] hit 16 distinct banks
    const int sr = lane & 15;
    const long long srow = i0 + sr;
    const float *grow = gI + (b * N + (srow < N ? srow : 0)) * T;
    float pv[8];
    auto prefetch = [&](int c) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long t = (long long)c * LCH + 4 * (4 * warp + 2 * h + (lane >> 4));
            if (VG) {
                float4 u = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (srow < N && t < T) u = __ldg(reinterpret_cast<const float4 *>(grow + t));
                pv[4 * h] = u.x; pv[4 * h + 1] = u.y; pv[4 * h + 2] = u.z; pv[4 * h + 3] = u.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) pv[4 * h + i] = (srow < N && t + i < T) ? __ldg(grow + t + i) : 0.0f;
            }
        }
    };
    float acc[LR];
#pragma unroll
    for (int r = 0; r < LR; ++r) acc[r] = 0.0f;
    float bsum = 0.0f;  // bias partial of row tid & 15, steps tid / 16 + 64 k of each chunk (z = 0 only)
    prefetch(0);
    if (VS) {  // chunk 0's words into slot 0
#pragma unroll
        for (int m = 0; m < LCW / 4; ++m) {
            const bool ok = jv && 4 * m < nwin;
            cp_async16_zfill(reinterpret_cast<uint4 *>(wsl) + slot_unit(tid, m), ok ? wrow + 4 * m : wrow, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int c = 0; c < nch; ++c) {
        // this chunk's spike words of input j (landed in slot c & 1; 0 past the raster, the last
        // word masked to T) and the mask of the nonzero ones; then the next chunk's copies go out
        uint32_t *slot = wsl + (size_t)(c & 1) * LCW * LTHREADS;
        if (VS) asm volatile("cp.async.wait_group 0;" ::: "memory");
        unsigned nzm = 0;
#pragma unroll
        for (int m = 0; m < LCW / 4; ++m) {
            uint4 u;
            if (VS) {
                u = reinterpret_cast<const uint4 *>(slot)[slot_unit(tid, m)];
            } else {
                u = make_uint4(0u, 0u, 0u, 0u);
                const int w0 = c * LCW + 4 * m;
                if (jv && w0 < nwin) u.x = __ldg(wrow + w0);
                if (jv && w0 + 1 < nwin) u.y = __ldg(wrow + w0 + 1);
                if (jv && w0 + 2 < nwin) u.z = __ldg(wrow + w0 + 2);
                if (jv && w0 + 3 < nwin) u.w = __ldg(wrow + w0 + 3);
            }
            if (c == nch - 1) {
                const int w0 = c * LCW + 4 * m;
                if (w0 == nwin - 1) u.x &= tail;
                if (w0 + 1 == nwin - 1) u.y &= tail;
                if (w0 + 2 == nwin - 1) u.z &= tail;
                if (w0 + 3 == nwin - 1) u.w &= tail;
            }
            if (!VS || c == nch - 1) reinterpret_cast<uint4 *>(slot)[slot_unit(tid, m)] = u;
            nzm |= ((u.x ? 1u : 0u) | (u.y ? 2u : 0u) | (u.z ? 4u : 0u) | (u.w ? 8u : 0u)) << (4 * m);
        }
        if (VS && c + 1 < nch) {
            uint32_t *nslot = wsl + (size_t)((c + 1) & 1) * LCW * LTHREADS;
#pragma unroll
            for (int m = 0; m < LCW / 4; ++m) {
                const int w0 = (c + 1) * LCW + 4 * m;
                const bool ok = jv && w0 < nwin;
                cp_async16_zfill(reinterpret_cast<uint4 *>(nslot) + slot_unit(tid, m), ok ? wrow + w0 : wrow, ok);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        __syncthreads();  // every thread is done with the previous chunk's gt
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = 4 * (4 * warp + 2 * h + (lane >> 4));
#pragma unroll
            for (int i = 0; i < 4; ++i) gt[(t + i) * LGS + sr] = pv[4 * h + i];
        }
        if (c + 1 < nch) prefetch(c + 1);
        __syncthreads();  // chunk c staged
        if (blockIdx.z == 0) {
#pragma unroll
            for (int k = 0; k < LCH / 64; ++k) bsum += gt[((tid >> 4) + 64 * k) * LGS + (tid & 15)];
        }
        // this input's spikes in step order, one per iteration across the warp
        uint32_t m = 0;
        int base = 0;
        while (__any_sync(FULL, m != 0u || nzm != 0u)) {
            if (m == 0u && nzm != 0u) {
                const int k = __ffs(nzm) - 1;
                nzm &= nzm - 1u;
                m = slot[4 * slot_unit(tid, k >> 2) + (k & 3)];
                base = 32 * k;
            }
            if (m != 0u) {
                const int t = base + __ffs(m) - 1;
                m &= m - 1u;
                const float4 *gp = reinterpret_cast<const float4 *>(gt + t * LGS);
#pragma unroll
                for (int q = 0; q < LR / 4; ++q) {
                    const float4 u = gp[q];
                    acc[4 * q] += u.x;
                    acc[4 * q + 1] += u.y;
                    acc[4 * q + 2] += u.z;
                    acc[4 * q + 3] += u.w;
                }
            }
        }
    }
    if (jv) {
#pragma unroll
        for (int r = 0; r < LR; ++r)
            if (i0 + r < N) part[(b * N + i0 + r) * ldp + j] = acc[r];
    }
    if (blockIdx.z == 0) {
        bsm[(tid >> 4) * LR + (tid & 15)] = bsum;
        __syncthreads();
        if (tid < LR && i0 + tid < N) {
            float s = 0.0f;
            for (int q = 0; q < 64; ++q) s += bsm[q * LR + tid];
            part_b[b * N + i0 + tid] = s;
        }
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
        static bool attr = false;
        const auto kernel_for = [](bool vg, bool vs) {
            return vg ? (vs ? gw_lane_kernel<true, true> : gw_lane_kernel<true, false>)
                      : (vs ? gw_lane_kernel<false, true> : gw_lane_kernel<false, false>);
        };
        if (!attr) {
            for (int v = 0; v < 4; ++v)
                if (cudaFuncSetAttribute(kernel_for(v & 1, v & 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)LSMEM) != cudaSuccess)
                    return (int)cudaGetLastError();
            attr = true;
        }
        const int nwin = (int)((T + 31) / 32);
        auto a16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
        const bool vg = (T % 4 == 0) && a16(gI), vs = (nwin % 4 == 0) && a16(S);
        const dim3 grid((unsigned)((N + LR - 1) / LR), (unsigned)B, (unsigned)((Nin + LJ - 1) / LJ));
        long long aN = N, aNin = Nin, aT = T;
        int anwin = nwin, aldp = ldp;
        void *args[] = {(void *)&gI, (void *)&S, &aN, &aNin, &aT, &anwin, &aldp, &part, &part_b};
        cudaError_t e = cudaLaunchKernel((const void *)kernel_for(vg, vs), grid, dim3(LTHREADS), args, LSMEM, stream);
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
