// Synaptic projection on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Feedforward input current of Eq 3 / Prop 3 for a batch of binary spike
// rasters:  I[b, i, t] = bias_i + sum_j W[i, j] S[b, j, t].
// Per batch element this is the GEMM D[N x T] = W[N x Nin] * S_b[Nin x T].
// W is carried as two BF16 terms (W = W_hi + W_lo up to 2^-16 |W|); spikes
// are exactly 0/1 in BF16, so each product is exact and the FP32 accumulator
// sees W_hi[i,j] + W_lo[i,j] for every active input.
//
// Tile: 128 neurons x 256 time steps (one tcgen05.mma M=128, N=256, K=16
// instruction shape).  The kernel is persistent (one CTA per SM walking the
// tiles) and warp-specialised: a TMA warp, an MMA warp, 4 builder warps and
// 4 epilogue warps coordinate through mbarriers; two TMEM accumulators (2 x
// 256 columns) let one tile's epilogue overlap the next tile's main loop.
// K runs over the inputs in slabs of 64 (one 128-byte swizzle atom of BF16):
//   * the TMA warp loads each slab's spike words (64 inputs x 256 steps = 2 KB
//     of bits) and its W_hi / W_lo tiles (cp.async.bulk.tensor, 128B swizzle)
//     into a 4-stage ring, words and weights on separate barriers so that the
//     builders can start as soon as the bits have landed (when the raster's row
//     pitch does not allow TMA, the builders read the words from global memory);
//   * 4 builder warps turn the bits into the BF16 spike slab [256 t x 64 j] of
//     a 2-stage ring: each warp owns 32 inputs x 4 time words (one 16-byte
//     shared load per lane), transposes 32x32 bit blocks with shuffles, expands
//     bit pairs to BF16 pairs arithmetically and stores 16-byte chunks in the
//     same 128B-swizzled K-major layout;
//   * the MMA warp's elected lane issues 8 MMAs per slab (4 K-steps x
//     {hi, lo}) and commits them to the weight stage's and the spike slab's
//     "free" barriers.
// Epilogue (4 warps, TMEM lanes 32w..32w+31): tcgen05.ld of 32 columns at a
// time, + bias, FP32 stores, then the accumulator is handed back to the MMA
// warp.  Every wait is bounded; a timeout sets a shared abort flag, every role
// leaves its loop, and the teardown waits (bounded) for copies and MMAs still
// in flight before TMEM is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstring>

#include "common.cuh"
#include "tmap.h"
#include "umma.cuh"

namespace alif {
namespace proj {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int NA = 4;  // weight (+ spike word) stages, filled by TMA
constexpr int NB = 2;  // spike-slab stages, built by the builder warps
constexpr int EPI_WARPS = 4, BUILD_WARPS = 4;
constexpr int TMA_WARP = EPI_WARPS + BUILD_WARPS, MMA_WARP = TMA_WARP + 1;
constexpr int THREADS = (MMA_WARP + 1) * 32;  // 320
constexpr int A_BYTES = BM * BK * 2;                 // 16 KB per weight term
constexpr int AST_BYTES = 2 * A_BYTES;               // hi + lo
constexpr int B_BYTES = BN * BK * 2;                 // 32 KB spike slab
constexpr int WORD_BYTES = BK * (BN / 32) * 4;       // 2 KB of spike bits
constexpr int OFF_B = NA * AST_BYTES;                // 128 KB
constexpr int OFF_W = OFF_B + NB * B_BYTES;          // 192 KB
constexpr int OFF_BAR = OFF_W + NA * WORD_BYTES;     // 200 KB
static_assert(AST_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "operand stages keep 1024-byte alignment");
constexpr int OFF_EPI = OFF_BAR + 256;               // per epilogue warp: a 32 x 32 output chunk
constexpr int EPI_STRIDE = 36;                        // floats per staged row (16-byte rows, no conflicts)
constexpr int EPI_BYTES = 32 * EPI_STRIDE * 4;        // 4.5 KB per epilogue warp
constexpr int SMEM_BYTES = OFF_EPI + EPI_WARPS * EPI_BYTES + 1024;  // + alignment slack
constexpr uint32_t TMEM_COLS = 512;  // two accumulators of 256 columns

struct Args {
    long long B, Nin, N, T, nwin, ldw;
    const uint32_t *S;
    const float *bias;
    float *I;
    int tiles_m, tiles_t, nk;
    long long tiles;
    int *status;
};

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = umma::idesc_bf16(BM, BN);
using umma::sw128_desc;
using umma::tma_load_2d;
using umma::mma_commit;
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    umma::mma_bf16(d, a, b, IDESC, acc);
}
__device__ __forceinline__ void tc_fence_before() { umma::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { umma::fence_after(); }

template <bool WORDS_TMA>
__global__ void __launch_bounds__(THREADS, 1)
    proj_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                const __grid_constant__ CUtensorMap tm_s, const Args A) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sm = smem_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
    uint64_t *a_full = bars;                   // [NA] weight slab landed (TMA tx)
    uint64_t *w_full = bars + NA;              // [NA] spike words landed (TMA tx)
    uint64_t *a_free = bars + 2 * NA;          // [NA] MMAs reading the weight stage completed
    uint64_t *b_full = bars + 3 * NA;          // [NB] spike slab built (4 builder warps)
    uint64_t *b_free = bars + 3 * NA + NB;     // [NB] MMAs reading the spike slab completed
    uint64_t *acc_full = bars + 3 * NA + 2 * NB;      // [2] tile accumulated
    uint64_t *acc_free = acc_full + 2;                // [2] tile read out (4 epilogue warps)
    uint64_t *drain = acc_full + 4;                   // [1] every MMA of this CTA completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_full + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    static_assert((3 * NA + 2 * NB + 5) * 8 + 8 <= 256, "barrier area");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&w_full[s], 1);
            mbar_init(&a_free[s], 1);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(&b_full[s], BUILD_WARPS);
            mbar_init(&b_free[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_free[q], EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
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
    const int nk = A.nk;
    auto tile_coords = [&](long long tile, int &m0, long long &t0, long long &b) {
        const int mt = (int)(tile % A.tiles_m);
        const long long rest = tile / A.tiles_m;
        m0 = mt * BM;
        t0 = (rest % A.tiles_t) * BN;
        b = rest / A.tiles_t;
    };
    auto fail = [&]() {
        report_timeout(A.status);
        *abort_flag = 1;
    };

    long long tma_issued = 0;  // TMA lane: slabs issued (weight stage g % NA for the g-th)
    if (warp == TMA_WARP) {
        // ---- loads: spike words, then the weight slab, NA slabs ahead of the MMAs
        if (lane == 0) {
            long long &g = tma_issued;
            for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x) {
                int m0;
                long long t0, b;
                tile_coords(tile, m0, t0, b);
                for (int kt = 0; kt < nk && !*abort_flag; ++kt, ++g) {
                    const int s = (int)(g % NA);
                    const long long n = g / NA;
                    if (n > 0 && !mbar_wait_bounded(&a_free[s], (uint32_t)((n - 1) & 1))) {
                        fail();
                        break;
                    }
                    if (WORDS_TMA) {
                        mbar_arrive_expect_tx(&w_full[s], WORD_BYTES);
                        tma_load_2d(base + OFF_W + s * WORD_BYTES, &tm_s, (int)(t0 >> 5),
                                    (int)(b * A.Nin + (long long)kt * BK), smem_u32(&w_full[s]));
                    }
                    const uint32_t st = base + s * AST_BYTES;
                    mbar_arrive_expect_tx(&a_full[s], AST_BYTES);
                    tma_load_2d(st, &tm_hi, kt * BK, m0, smem_u32(&a_full[s]));
                    tma_load_2d(st + A_BYTES, &tm_lo, kt * BK, m0, smem_u32(&a_full[s]));
                }
                if (*abort_flag) break;
            }
        }
    } else if (warp == MMA_WARP) {
        // ---- tensor core: 8 MMAs per slab into the tile's accumulator
        if (lane == 0) {
            long long g = 0, it = 0;
            for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x, ++it) {
                const int buf = (int)(it & 1);
                const uint32_t dacc = tmem + (uint32_t)(buf * 256);
                if (it >= 2 && !mbar_wait_bounded(&acc_free[buf], (uint32_t)(((it >> 1) - 1) & 1))) {
                    fail();
                    break;
                }
                tc_fence_after();
                for (int kt = 0; kt < nk; ++kt, ++g) {
                    const int sa = (int)(g % NA), sb = (int)(g % NB);
                    if (!mbar_wait_bounded(&a_full[sa], (uint32_t)((g / NA) & 1)) ||
                        !mbar_wait_bounded(&b_full[sb], (uint32_t)((g / NB) & 1))) {
                        fail();
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_hi = base + sa * AST_BYTES, a_lo = a_hi + A_BYTES, b_sm = base + OFF_B + sb * B_BYTES;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t bd = sw128_desc(b_sm + ks * 32);
                        mma_bf16(dacc, sw128_desc(a_hi + ks * 32), bd, (kt > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(dacc, sw128_desc(a_lo + ks * 32), bd, 1u);
                    }
                    mma_commit(smem_u32(&a_free[sa]));  // weight stage reusable once these MMAs finish
                    mma_commit(smem_u32(&b_free[sb]));  // spike slab likewise
                }
                if (*abort_flag) break;
                mma_commit(smem_u32(&acc_full[buf]));  // tile complete
            }
        }
    } else if (warp >= EPI_WARPS) {
        // ---- builders: spike slab rows t (0..255), 64 BF16 inputs per row, 128B swizzle.
        // Builder warp bw owns inputs jh*32.. (jh = bw / 2) at time words tb0..tb0+3
        // (tb0 = 4 (bw % 2)): one 16-byte shared load per lane brings its input's 4 words.
        const int bw = warp - EPI_WARPS;
        const int jh = bw >> 1, tb0 = 4 * (bw & 1);
        long long g = 0;
        for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x) {
            int m0;
            long long t0, b;
            tile_coords(tile, m0, t0, b);
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int sa = (int)(g % NA), sb = (int)(g % NB);
                const long long nbu = g / NB;
                if ((WORDS_TMA && !mbar_wait_bounded(&w_full[sa], (uint32_t)((g / NA) & 1))) ||
                    (nbu > 0 && !mbar_wait_bounded(&b_free[sb], (uint32_t)((nbu - 1) & 1)))) {
                    fail();
                    break;
                }
                unsigned char *bs = sm + OFF_B + sb * B_BYTES;
                const long long j = (long long)kt * BK + jh * 32 + lane;
                const long long tw0 = (t0 >> 5) + tb0;
                uint32_t wv[4] = {0u, 0u, 0u, 0u};
                if (j < A.Nin) {
                    if (WORDS_TMA) {
                        const uint4 u = *reinterpret_cast<const uint4 *>(sm + OFF_W + sa * WORD_BYTES +
                                                                         ((jh * 32 + lane) * (BN / 32) + tb0) * 4);
                        wv[0] = u.x; wv[1] = u.y; wv[2] = u.z; wv[3] = u.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (tw0 + q < A.nwin) wv[q] = __ldg(A.S + (b * A.Nin + j) * A.nwin + tw0 + q);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (tw0 + q >= A.nwin) wv[q] = 0u;
                        if (tw0 + q == A.nwin - 1 && (A.T & 31)) wv[q] &= (1u << (A.T & 31)) - 1u;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int tb = tb0 + q;
                    const uint32_t y = bits_transpose32(wv[q], lane);  // inputs jh*32.. at step tb*32 + lane
                    const int row = tb * 32 + lane;
                    unsigned char *rp = bs + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        // bits 2m, 2m+1 of y -> BF16 pair (1.0 where set): low half
                        // bit(2m) * 0x3F80, high half bit(2m+1) * 0x3F80
                        uint32_t wq[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int m = 4 * c4 + e;
                            const uint32_t z = (y >> (2 * m)) & 3u;
                            wq[e] = z * 0x3F80u + (z >> 1) * 0x3F7F8100u;
                        }
                        const int chunk = (jh * 4 + c4) ^ (row & 7);
                        *reinterpret_cast<uint4 *>(rp + chunk * 16) = make_uint4(wq[0], wq[1], wq[2], wq[3]);
                    }
                }
                fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&b_full[sb]);
            }
            if (*abort_flag) break;
        }
    } else {
        // ---- epilogue warps: TMEM lanes 32 w .. 32 w + 31 = neuron rows of the tile
        long long it = 0;
        const bool vec = ((A.T & 3) == 0) && ((reinterpret_cast<uintptr_t>(A.I) & 15u) == 0);
        for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x, ++it) {
            int m0;
            long long t0, b;
            tile_coords(tile, m0, t0, b);
            const int buf = (int)(it & 1);
            if (!mbar_wait_bounded(&acc_full[buf], (uint32_t)((it >> 1) & 1))) {
                fail();
                break;
            }
            tc_fence_after();
            const int row = m0 + warp * 32 + lane;
            const float bias = (A.bias && row < A.N) ? A.bias[row] : 0.0f;
            float *out = A.I + (b * A.N + row) * A.T;
            // Each 32 x 32 chunk (lane = row) goes through this warp's staging area so
            // that every store instruction writes 4 whole 128-byte row segments: lane L
            // stores row 4 i + L / 8, columns 4 (L % 8) .. + 3.
            float *stage = reinterpret_cast<float *>(sm + OFF_EPI + warp * EPI_BYTES);
            const int srow = lane >> 3, scol = 4 * (lane & 7);
            const long long row0 = (long long)m0 + warp * 32;  // first row of this warp's 32
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 256 + c * 32);
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
                const long long c0 = t0 + c * 32;
                if (vec && c0 + 32 <= A.T) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4 *>(stage + lane * EPI_STRIDE + 4 * q) = make_float4(
                            __uint_as_float(r[4 * q]) + bias, __uint_as_float(r[4 * q + 1]) + bias,
                            __uint_as_float(r[4 * q + 2]) + bias, __uint_as_float(r[4 * q + 3]) + bias);
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int rr = 4 * i + srow;
                        const float4 v = *reinterpret_cast<const float4 *>(stage + rr * EPI_STRIDE + scol);
                        if (row0 + rr < A.N)
                            *reinterpret_cast<float4 *>(A.I + (b * A.N + row0 + rr) * A.T + c0 + scol) = v;
                    }
                    __syncwarp();  // the staging area is rewritten by the next chunk
                } else if (row < A.N) {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (c0 + q < A.T) out[c0 + q] = __uint_as_float(r[q]) + bias;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_free[buf]);
        }
    }
    // Teardown.  No copy may still be landing in shared memory, no MMA still
    // writing TMEM and no commit still arriving on a barrier when the CTA
    // exits: the TMA lane waits (bounded) for its last loads on every stage
    // and, after a clean run, for the MMAs' release of every weight stage; the
    // MMA lane commits once more and waits for that commit.
    if (warp == TMA_WARP && lane == 0) {
        const long long issued = tma_issued;
        for (int s = 0; s < NA && s < issued; ++s) {
            const uint32_t par = (uint32_t)(((issued - 1 - s) / NA) & 1);
            (void)mbar_wait_bounded(&a_full[s], par, 100000000ull);
            if (WORDS_TMA) (void)mbar_wait_bounded(&w_full[s], par, 100000000ull);
            if (!*abort_flag) (void)mbar_wait_bounded(&a_free[s], par, 100000000ull);
        }
    }
    if (warp == MMA_WARP && lane == 0) {
        mma_commit(smem_u32(drain));
        (void)mbar_wait_bounded(drain, 0u, 100000000ull);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
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
int make_map(CUtensorMap *map, const uint16_t *W, long long N, long long ldw) {
    const auto g_encode = tensor_map_encoder();
    if (!g_encode) return -1;
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
    const auto g_encode = tensor_map_encoder();
    if (!g_encode) return -1;
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
    A.tiles = tiles;
    if (tiles == 0) return 0;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
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
        proj_kernel<true><<<grid, THREADS, SMEM_BYTES, stream>>>(mh, ml, ms, A);
    else
        proj_kernel<false><<<grid, THREADS, SMEM_BYTES, stream>>>(mh, ml, ms, A);
    return (int)cudaGetLastError();
}

}  // namespace alif
