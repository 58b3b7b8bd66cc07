// Synaptic projection on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Feedforward input current of Eq 3 / Prop 3 for a batch of binary spike
// rasters:  I[b, i, t] = bias_i + sum_j W[i, j] S[b, j, t].
// Per batch element this is the GEMM D[N x T] = W[N x Nin] * S_b[Nin x T].
// W is carried as two BF16 terms (W = W_hi + W_lo up to 2^-16 |W|); spikes
// are exactly 0/1 in BF16, so each product is exact and the FP32 accumulator
// sees W_hi[i,j] + W_lo[i,j] for every active input.
//
// Tile: 128 neurons x 256 time steps per CTA (one tcgen05.mma M=128, N=256,
// K=16 instruction shape), accumulator in TMEM (256 columns).  K runs over
// the inputs in slabs of 64 (one 128-byte swizzle atom of BF16):
//   * W_hi / W_lo slabs arrive by TMA (cp.async.bulk.tensor, 128B swizzle);
//   * the slab's spike words (64 inputs x 256 steps = 2 KB of bits) arrive by
//     TMA too (when the raster's row pitch allows it, else by plain loads);
//   * the spike slab [256 t x 64 j] is built by the CTA's threads from those
//     bits: each warp transposes 32x32 bit blocks with shuffles, expands
//     bytes to BF16 through a 256-entry table and stores 16-byte chunks in
//     the same 128B-swizzled K-major layout;
//   * one thread issues 8 MMAs per slab (4 K-steps x {hi, lo}) and commits
//     them to an mbarrier; a 3-stage ring keeps the loads two slabs ahead.
// Epilogue: tcgen05.ld of 32 columns at a time, + bias, FP32 stores.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstring>

#include "common.cuh"

namespace alif {
namespace proj {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int STAGES = 3;
constexpr int THREADS = 128;
constexpr int A_BYTES = BM * BK * 2;                 // 16 KB per weight term
constexpr int B_BYTES = BN * BK * 2;                 // 32 KB spike slab
constexpr int WORD_BYTES = BK * (BN / 32) * 4;       // 2 KB of spike bits
constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES + WORD_BYTES;  // 66 KB (multiple of 1024)
static_assert(STAGE_BYTES % 1024 == 0, "stages must keep 1024-byte alignment");
constexpr int LUT_BYTES = 256 * 16;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + LUT_BYTES + 256 + 1024;  // + barriers + align
constexpr uint32_t TMEM_COLS = 256;

struct Args {
    long long B, Nin, N, T, nwin, ldw;
    const uint32_t *S;
    const float *bias;
    float *I;
    int tiles_m, tiles_t, nk;
    int *status;
};

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 x 32 bit-matrix transpose across the warp (recursive block swap):
// in: lane r holds row r (bit c = A[r][c]); out: lane r holds column r.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const int j = 16 >> l;
        const uint32_t m = masks[l];
        const uint32_t y = __shfl_xor_sync(FULL, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

template <bool WORDS_TMA>
__global__ void __launch_bounds__(THREADS, 1)
    proj_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                const __grid_constant__ CUtensorMap tm_s, const Args A) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sm = smem_raw + (base - raw);
    uint4 *lut = reinterpret_cast<uint4 *>(sm + STAGES * STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + STAGES * STAGE_BYTES + LUT_BYTES);
    uint64_t *tma_full = bars;          // [STAGES]
    uint64_t *mma_done = bars + STAGES;  // [STAGES]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile order: the 8 neuron tiles of one (b, t-range) are adjacent (spike slab reuse in L2)
    const long long tile = blockIdx.x;
    const int mt = (int)(tile % A.tiles_m);
    const long long rest = tile / A.tiles_m;
    const int tt = (int)(rest % A.tiles_t);
    const long long b = rest / A.tiles_t;
    const int m0 = mt * BM;
    const long long t0 = (long long)tt * BN;

    // expansion table: byte e -> 8 BF16 values (1.0 where bit set)
    for (int e = tid; e < 256; e += THREADS) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            w[q] = (((e >> (2 * q)) & 1) ? 0x3F80u : 0u) | (((e >> (2 * q + 1)) & 1) ? 0x3F800000u : 0u);
        lut[e] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&tma_full[s], 1);
            mbar_init(&mma_done[s], 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // Every thread reaches every barrier: a timed-out wait only clears `ok`,
    // which the CTA agrees on (__syncthreads_and) before acting on it.
    bool ok = true;
    const int nk = A.nk;
    int committed = -1;  // last slab whose MMAs were committed (thread 0)
    const uint32_t tx = 2 * A_BYTES + (WORDS_TMA ? WORD_BYTES : 0);
    auto issue_loads = [&](int k) {  // thread 0: weights (+ spike words) of slab k into its stage
        const int s = k % STAGES;
        const uint32_t st_base = base + s * STAGE_BYTES;
        mbar_arrive_expect_tx(&tma_full[s], tx);
        tma_load_2d(st_base, &tm_hi, k * BK, m0, smem_u32(&tma_full[s]));
        tma_load_2d(st_base + A_BYTES, &tm_lo, k * BK, m0, smem_u32(&tma_full[s]));
        if (WORDS_TMA)
            tma_load_2d(st_base + 2 * A_BYTES + B_BYTES, &tm_s, (int)(t0 >> 5), (int)(b * A.Nin + (long long)k * BK),
                        smem_u32(&tma_full[s]));
    };
    if (tid == 0)
        for (int k = 0; k < STAGES && k < nk; ++k) issue_loads(k);
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int s = kt % STAGES;
        unsigned char *st = sm + s * STAGE_BYTES;
        const uint32_t a_hi = base + s * STAGE_BYTES, a_lo = a_hi + A_BYTES, b_sm = a_hi + 2 * A_BYTES;
        const uint32_t *words = reinterpret_cast<const uint32_t *>(st + 2 * A_BYTES + B_BYTES);
        if (!mbar_wait_bounded(&tma_full[s], (kt / STAGES) & 1u)) {
            report_timeout(A.status);
            ok = false;
        }
        ok = __syncthreads_and(ok);
        if (!ok) break;  // uniform across the CTA
        // spike slab: rows t (0..255), 64 BF16 inputs per row, 128B swizzle
        {
            unsigned char *bs = st + 2 * A_BYTES;
            const long long j0 = (long long)kt * BK;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int blk = warp + 4 * q;  // 16 blocks of 32 inputs x 32 steps
                const int jh = blk >> 3, tb = blk & 7;
                const long long j = j0 + jh * 32 + lane;
                const long long tw = (t0 >> 5) + tb;
                uint32_t x = 0;
                if (j < A.Nin && tw < A.nwin) {
                    x = WORDS_TMA ? words[(jh * 32 + lane) * (BN / 32) + tb]
                                  : __ldg(A.S + (b * A.Nin + j) * A.nwin + tw);
                    if (tw == A.nwin - 1 && (A.T & 31)) x &= (1u << (A.T & 31)) - 1u;
                }
                const uint32_t y = transpose32(x, lane);  // inputs jh*32.. at step tb*32 + lane
                const int row = tb * 32 + lane;
                unsigned char *rp = bs + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int chunk = (jh * 4 + c4) ^ (row & 7);
                    *reinterpret_cast<uint4 *>(rp + chunk * 16) = lut[(y >> (8 * c4)) & 0xFFu];
                }
            }
        }
        fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t bd = sw128_desc(b_sm + ks * 32);
                mma_bf16(tmem, sw128_desc(a_hi + ks * 32), bd, (kt > 0 || ks > 0) ? 1u : 0u);
                mma_bf16(tmem, sw128_desc(a_lo + ks * 32), bd, 1u);
            }
            mma_commit(smem_u32(&mma_done[s]));
            committed = kt;
            // refill the stage of slab kt-1 with slab kt-1+STAGES once its MMAs are done
            const int kp = kt - 1, kn = kt - 1 + STAGES;
            if (kp >= 0 && kn < nk) {
                if (mbar_wait_bounded(&mma_done[kp % STAGES], (kp / STAGES) & 1u)) {
                    issue_loads(kn);
                } else {
                    report_timeout(A.status);
                    ok = false;
                }
            }
        }
        ok = __syncthreads_and(ok);
    }
    if (tid == 0) *reinterpret_cast<int *>(tmem_slot + 1) = committed;
    __syncthreads();
    committed = *reinterpret_cast<int *>(tmem_slot + 1);

    // Wait for the last committed slab (MMAs complete in issue order); this
    // also drains the tensor core before TMEM is read or released.
    bool acc_ready = false;
    if (committed >= 0) {
        acc_ready = mbar_wait_bounded(&mma_done[committed % STAGES], (committed / STAGES) & 1u);
        if (!acc_ready) report_timeout(A.status);
    }
    acc_ready = __syncthreads_and(acc_ready && ok && committed == nk - 1);
    tc_fence_after();

    if (acc_ready) {
        const int row = m0 + warp * 32 + lane;
        const float bias = (A.bias && row < A.N) ? A.bias[row] : 0.0f;
        float *out = A.I + (b * A.N + row) * A.T;
        const bool vec = ((A.T & 3) == 0) && ((reinterpret_cast<uintptr_t>(A.I) & 15u) == 0);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < A.N) {
                const long long c0 = t0 + c * 32;
                if (vec && c0 + 32 <= A.T) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        reinterpret_cast<float4 *>(out + c0)[q] =
                            make_float4(__uint_as_float(r[4 * q]) + bias, __uint_as_float(r[4 * q + 1]) + bias,
                                        __uint_as_float(r[4 * q + 2]) + bias, __uint_as_float(r[4 * q + 3]) + bias);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (c0 + q < A.T) out[c0 + q] = __uint_as_float(r[q]) + bias;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

__global__ void split_pad_kernel(const float *W, long long N, long long Nin, long long ldw, uint16_t *hi,
                                 uint16_t *lo) {
    const long long total = N * ldw;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = k / ldw, j = k - i * ldw;
        uint16_t h = 0, l = 0;
        if (j < Nin) {
            const float w = W[i * Nin + j];
            const __nv_bfloat16 bh = __float2bfloat16_rn(w);
            h = __bfloat16_as_ushort(bh);
            l = __bfloat16_as_ushort(__float2bfloat16_rn(w - __bfloat162float(bh)));
        }
        hi[k] = h;
        lo[k] = l;
    }
}

}  // namespace proj

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int get_encode() {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return 0;
}

int make_map(CUtensorMap *map, const uint16_t *W, long long N, long long ldw) {
    if (get_encode()) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)ldw, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)ldw * 2};
    const cuuint32_t box[2] = {proj::BK, proj::BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(W), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

// Spike words [B*Nin rows, nwin words], box 8 words x 64 rows (no swizzle).
int make_words_map(CUtensorMap *map, const uint32_t *S, long long rows, long long nwin) {
    if (get_encode()) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)nwin, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)nwin * 4};
    const cuuint32_t box[2] = {proj::BN / 32, proj::BK};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t *>(S), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}
}  // namespace

int launch_split_pad(const float *W, long long N, long long Nin, long long ldw, uint16_t *hi, uint16_t *lo,
                     cudaStream_t stream) {
    const long long total = N * ldw;
    if (total == 0) return 0;
    long long blocks = (total + 255) / 256;
    if (blocks > 65535LL * 8) blocks = 65535LL * 8;
    proj::split_pad_kernel<<<(unsigned)blocks, 256, 0, stream>>>(W, N, Nin, ldw, hi, lo);
    return (int)cudaGetLastError();
}

// Returns 0, a CUDA error code (> 0), or -1/-2 when the tensor maps cannot be built.
int launch_syn_project(long long B, long long Nin, long long N, long long T, const uint16_t *W_hi,
                       const uint16_t *W_lo, long long ldw, const uint32_t *S, const float *bias, float *I,
                       int *status, cudaStream_t stream) {
    using namespace proj;
    CUtensorMap mh, ml;
    int rc = make_map(&mh, W_hi, N, ldw);
    if (rc) return rc;
    rc = make_map(&ml, W_lo, N, ldw);
    if (rc) return rc;
    Args A;
    A.B = B;
    A.Nin = Nin;
    A.N = N;
    A.T = T;
    A.nwin = (T + 31) / 32;
    A.ldw = ldw;
    A.S = S;
    A.bias = bias;
    A.I = I;
    A.tiles_m = (int)((N + BM - 1) / BM);
    A.tiles_t = (int)((T + BN - 1) / BN);
    A.nk = (int)((Nin + BK - 1) / BK);
    A.status = status;
    const long long tiles = (long long)A.tiles_m * A.tiles_t * B;
    if (tiles == 0) return 0;
    // spike words by TMA when the row pitch (nwin * 4 bytes) and base allow it
    CUtensorMap ms;
    const bool words_tma = (A.nwin % 4 == 0) && ((reinterpret_cast<uintptr_t>(S) & 15u) == 0) &&
                           make_words_map(&ms, S, B * Nin, A.nwin) == 0;
    if (!words_tma) memset(&ms, 0, sizeof ms);
    static bool attr[2] = {false, false};
    if (!attr[words_tma]) {
        if (words_tma)
            cudaFuncSetAttribute(proj_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        else
            cudaFuncSetAttribute(proj_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr[words_tma] = true;
    }
    if (words_tma)
        proj_kernel<true><<<(unsigned)tiles, THREADS, SMEM_BYTES, stream>>>(mh, ml, ms, A);
    else
        proj_kernel<false><<<(unsigned)tiles, THREADS, SMEM_BYTES, stream>>>(mh, ml, ms, A);
    return (int)cudaGetLastError();
}

}  // namespace alif
