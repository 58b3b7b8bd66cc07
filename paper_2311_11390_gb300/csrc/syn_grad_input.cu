// Input gradient of the synaptic projection on the tcgen05 tensor cores (sm_103a):
//     grad_S[b, j, t] = sum_i W[i, j] grad_I[b, i, t]
// the adjoint of the feedforward term of Eq 3 / Prop 3.  Per batch element it is the GEMM
// D[Nin x T] = W^T[Nin x N] * G_b[N x T], both operands FP32.  Each operand is split into two
// BF16 terms (x = x_hi + x_lo + r with |r| <= 2^-16 |x|, round-to-nearest-even), and three
// products, each exact in FP32, are accumulated in FP32 in TMEM: W_hi G_hi + W_hi G_lo +
// W_lo G_hi (the fourth, W_lo G_lo, is below 2^-16 of a product).  Per output the error against
// the exact sum is at most sum_i |W_ij| |G_i| (3 * 2^-16 + (3N + 2) 2^-24).
//
// Tile: 128 inputs j x 256 steps t, K over the neurons i in slabs of 64.  Persistent kernel
// (one CTA per SM walking the tiles, inputs fastest so that the CTAs working on one
// (batch, step) tile read the same G slab out of L2), warp-specialised like the projection:
//   * a TMA warp loads W^T's hi / lo slabs [128 j x 64 i] (128B swizzle, K-major) into a
//     2-stage ring;
//   * 8 converter warps read the FP32 slab G_b[64 i x 256 t] straight from global memory
//     (a warp reads 32 consecutive steps of one neuron per load, the next half slab's loads
//     issued before the current half is converted), split every value into its
//     two BF16 terms and store them transposed, one step per thread, as the K-major
//     [256 t x 64 i] hi and lo operands (same swizzled layout as the projection's spike slab)
//     of a 2-stage ring;
//   * the MMA warp's elected lane issues 12 MMAs per slab (4 K-steps x 3 products);
//   * 4 epilogue warps drain the two 256-column TMEM accumulators (one tile's epilogue
//     overlaps the next tile's products) through a staging area into row segments of
//     grad_S.
// Every wait is bounded; a timeout sets a shared abort flag, every role leaves its loop and
// the teardown waits (bounded) for copies and MMAs in flight before TMEM is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "common.cuh"
#include "tmap.h"
#include "umma.cuh"

namespace alif {
namespace gin {

constexpr int BM = 128;  // inputs j per tile (TMEM lanes)
constexpr int BN = 256;  // steps t per tile (TMEM columns)
constexpr int BK = 64;   // neurons i per slab (one 128-byte swizzle atom of BF16)
constexpr int NA = 2;    // W^T slab stages (TMA)
constexpr int NB = 2;    // G slab stages (converters)
constexpr int EPI_WARPS = 4, CONV_WARPS = 8;
constexpr int TMA_WARP = EPI_WARPS + CONV_WARPS, MMA_WARP = TMA_WARP + 1;
constexpr int THREADS = (MMA_WARP + 1) * 32;  // 448
constexpr int A_BYTES = BM * BK * 2;          // 16 KB per term
constexpr int AST_BYTES = 2 * A_BYTES;        // hi + lo
constexpr int B_BYTES = BN * BK * 2;          // 32 KB per term
constexpr int BST_BYTES = 2 * B_BYTES;        // hi + lo
constexpr int OFF_B = NA * AST_BYTES;         // 64 KB
constexpr int OFF_BAR = OFF_B + NB * BST_BYTES;  // 192 KB
static_assert(AST_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "operand stages keep 1024-byte alignment");
constexpr int OFF_EPI = OFF_BAR + 256;
constexpr int EPI_STRIDE = 36;  // floats per staged row (16-byte rows, no bank conflicts)
constexpr int EPI_BYTES = 32 * EPI_STRIDE * 4;
constexpr int SMEM_BYTES = OFF_EPI + EPI_WARPS * EPI_BYTES + 1024;  // + alignment slack
constexpr uint32_t TMEM_COLS = 512;                                 // two accumulators of 256 columns
constexpr uint32_t IDESC = umma::idesc_bf16(BM, BN);
static_assert(CONV_WARPS * 32 == BN, "one converter thread per step of the tile");

struct Args {
    long long B, N, Nin, T;
    const float *G;  // [B, N, T]
    float *out;      // [B, Nin, T]
    int tiles_m, tiles_t, nk;
    long long tiles;
    int *status;
};

// x -> (hi, lo) BF16 pairs for two values: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __float22bfloat162_rn(make_float2(a, b));
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(a - hf.x, b - hf.y));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__global__ void __launch_bounds__(THREADS, 1)
    gin_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, const Args A) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned swizzled tiles
    unsigned char *sm = smem_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
    uint64_t *a_full = bars;                  // [NA] W^T slab landed (TMA tx)
    uint64_t *a_free = bars + NA;             // [NA] MMAs reading it completed
    uint64_t *b_full = bars + 2 * NA;         // [NB] G slab converted (CONV_WARPS arrivals)
    uint64_t *b_free = bars + 2 * NA + NB;    // [NB] MMAs reading it completed
    uint64_t *acc_full = bars + 2 * NA + 2 * NB;  // [2] tile accumulated
    uint64_t *acc_free = acc_full + 2;            // [2] tile read out (EPI_WARPS arrivals)
    uint64_t *drain = acc_full + 4;               // every MMA of this CTA completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_full + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    static_assert((2 * NA + 2 * NB + 5) * 8 + 8 <= 256, "barrier area");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NA; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_free[s], 1);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(&b_full[s], CONV_WARPS);
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
    if (warp == 0) umma::tmem_alloc(tmem_slot, TMEM_COLS);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
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

    long long tma_issued = 0;
    if (warp == TMA_WARP) {
        // ---- W^T hi / lo slabs, NA ahead of the MMAs
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
                    const uint32_t st = base + s * AST_BYTES;
                    mbar_arrive_expect_tx(&a_full[s], AST_BYTES);
                    umma::tma_load_2d(st, &tm_hi, kt * BK, m0, smem_u32(&a_full[s]));
                    umma::tma_load_2d(st + A_BYTES, &tm_lo, kt * BK, m0, smem_u32(&a_full[s]));
                }
                if (*abort_flag) break;
            }
        }
    } else if (warp == MMA_WARP) {
        // ---- tensor core: 12 MMAs per slab into the tile's accumulator
        if (lane == 0) {
            long long g = 0, it = 0;
            for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x, ++it) {
                const int buf = (int)(it & 1);
                const uint32_t dacc = tmem + (uint32_t)(buf * BN);
                if (it >= 2 && !mbar_wait_bounded(&acc_free[buf], (uint32_t)(((it >> 1) - 1) & 1))) {
                    fail();
                    break;
                }
                umma::fence_after();
                for (int kt = 0; kt < nk; ++kt, ++g) {
                    const int sa = (int)(g % NA), sb = (int)(g % NB);
                    if (!mbar_wait_bounded(&a_full[sa], (uint32_t)((g / NA) & 1)) ||
                        !mbar_wait_bounded(&b_full[sb], (uint32_t)((g / NB) & 1))) {
                        fail();
                        break;
                    }
                    umma::fence_after();
                    const uint32_t a_hi = base + sa * AST_BYTES, a_lo = a_hi + A_BYTES;
                    const uint32_t b_hi = base + OFF_B + sb * BST_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t ah = umma::sw128_desc(a_hi + ks * 32), al = umma::sw128_desc(a_lo + ks * 32);
                        const uint64_t bh = umma::sw128_desc(b_hi + ks * 32), bl = umma::sw128_desc(b_lo + ks * 32);
                        umma::mma_bf16(dacc, ah, bh, IDESC, (kt > 0 || ks > 0) ? 1u : 0u);
                        umma::mma_bf16(dacc, ah, bl, IDESC, 1u);
                        umma::mma_bf16(dacc, al, bh, IDESC, 1u);
                    }
                    umma::mma_commit(smem_u32(&a_free[sa]));
                    umma::mma_commit(smem_u32(&b_free[sb]));
                }
                if (*abort_flag) break;
                umma::mma_commit(smem_u32(&acc_full[buf]));
            }
        }
    } else if (warp >= EPI_WARPS) {
        // ---- converters: step row = (warp - EPI_WARPS) * 32 + lane of the slab, 64 neurons in two
        // halves of 32.  The loads of the next half (next slab, next tile) are issued before the
        // current half is converted, so that global-memory latency overlaps the conversion.
        const int row = (warp - EPI_WARPS) * 32 + lane;
        auto fetch = [&](float (&x)[32], long long tile, int kt, int half) {
            int m0;
            long long t0, b;
            tile_coords(tile, m0, t0, b);
            const long long t = t0 + row;
            const long long i0 = (long long)kt * BK + half * 32;
            const float *gp = A.G + (b * A.N + i0) * A.T + t;
#pragma unroll
            for (int e = 0; e < 32; ++e)
                x[e] = (t < A.T && i0 + e < A.N) ? __ldg(gp + (long long)e * A.T) : 0.0f;
        };
        float nx[32];
        if (blockIdx.x < A.tiles) fetch(nx, blockIdx.x, 0, 0);
        long long g = 0;
        for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x) {
            for (int kt = 0; kt < nk; ++kt, ++g) {
                const int sb = (int)(g % NB);
                const long long nbu = g / NB;
                if (nbu > 0 && !mbar_wait_bounded(&b_free[sb], (uint32_t)((nbu - 1) & 1))) {
                    fail();
                    break;
                }
                unsigned char *rh = sm + OFF_B + sb * BST_BYTES + (row >> 3) * 1024 + (row & 7) * 128;
                unsigned char *rl = rh + B_BYTES;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float x[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) x[e] = nx[e];
                    // prefetch the next half: this slab's second, else the next slab's (or tile's) first
                    if (half == 0)
                        fetch(nx, tile, kt, 1);
                    else if (kt + 1 < nk)
                        fetch(nx, tile, kt + 1, 0);
                    else if (tile + gridDim.x < A.tiles)
                        fetch(nx, tile + gridDim.x, 0, 0);
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {  // 8 neurons per 16-byte chunk
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) split2(x[8 * c4 + 2 * e], x[8 * c4 + 2 * e + 1], h[e], l[e]);
                        const int chunk = (half * 4 + c4) ^ (row & 7);
                        *reinterpret_cast<uint4 *>(rh + chunk * 16) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4 *>(rl + chunk * 16) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                }
                fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&b_full[sb]);
            }
            if (*abort_flag) break;
        }
    } else {
        // ---- epilogue warps: TMEM lanes 32 w .. 32 w + 31 = input rows of the tile
        long long it = 0;
        const bool vec = ((A.T & 3) == 0) && ((reinterpret_cast<uintptr_t>(A.out) & 15u) == 0);
        float *stage = reinterpret_cast<float *>(sm + OFF_EPI + warp * EPI_BYTES);
        const int srow = lane >> 3, scol = 4 * (lane & 7);
        for (long long tile = blockIdx.x; tile < A.tiles && !*abort_flag; tile += gridDim.x, ++it) {
            int m0;
            long long t0, b;
            tile_coords(tile, m0, t0, b);
            const int buf = (int)(it & 1);
            if (!mbar_wait_bounded(&acc_full[buf], (uint32_t)((it >> 1) & 1))) {
                fail();
                break;
            }
            umma::fence_after();
            const long long row0 = (long long)m0 + warp * 32;  // first input row of this warp
            const long long row = row0 + lane;
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * BN + c * 32), r);
                const long long c0 = t0 + c * 32;
                if (vec && c0 + 32 <= A.T) {
                    // through the staging area, so that each store writes 4 whole 128-byte row segments
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4 *>(stage + lane * EPI_STRIDE + 4 * q) =
                            make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                        __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int rr = 4 * i + srow;
                        const float4 v = *reinterpret_cast<const float4 *>(stage + rr * EPI_STRIDE + scol);
                        if (row0 + rr < A.Nin)
                            *reinterpret_cast<float4 *>(A.out + (b * A.Nin + row0 + rr) * A.T + c0 + scol) = v;
                    }
                    __syncwarp();  // the staging area is rewritten by the next chunk
                } else if (row < A.Nin) {
                    float *o = A.out + (b * A.Nin + row) * A.T;
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (c0 + q < A.T) o[c0 + q] = __uint_as_float(r[q]);
                }
            }
            umma::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_free[buf]);
        }
    }
    // Teardown: no copy may still be landing in shared memory, no MMA still writing TMEM and
    // no commit still arriving on a barrier when the CTA exits.
    if (warp == TMA_WARP && lane == 0) {
        const long long issued = tma_issued;
        for (int s = 0; s < NA && s < issued; ++s) {
            const uint32_t par = (uint32_t)(((issued - 1 - s) / NA) & 1);
            (void)mbar_wait_bounded(&a_full[s], par, 100000000ull);
            if (!*abort_flag) (void)mbar_wait_bounded(&a_free[s], par, 100000000ull);
        }
    }
    if (warp == MMA_WARP && lane == 0) {
        umma::mma_commit(smem_u32(drain));
        (void)mbar_wait_bounded(drain, 0u, 100000000ull);
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    if (warp == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// W [N, Nin] FP32 -> W^T split into BF16 terms, [Nin, ldk] each, zero beyond N.
__global__ void wt_split_kernel(const float *W, long long N, long long Nin, long long ldk, uint16_t *hi,
                                uint16_t *lo) {
    const long long total = Nin * ldk;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long j = k / ldk, i = k - j * ldk;
        uint16_t h = 0, l = 0;
        if (i < N) {
            const float w = W[i * Nin + j];
            const __nv_bfloat16 bh = __float2bfloat16_rn(w);
            h = __bfloat16_as_ushort(bh);
            l = __bfloat16_as_ushort(__float2bfloat16_rn(w - __bfloat162float(bh)));
        }
        hi[k] = h;
        lo[k] = l;
    }
}

int make_wt_map(CUtensorMap *map, const uint16_t *Wt, long long Nin, long long ldk) {
    const auto enc = tensor_map_encoder();
    if (!enc) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)Nin};
    const cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
    const cuuint32_t box[2] = {BK, BM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(Wt), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace gin

// Bytes of scratch the input gradient needs: the two BF16 terms of W^T, [Nin, ldk] each.
size_t syn_grad_input_ws(long long N, long long Nin) {
    const long long ldk = (N + gin::BK - 1) / gin::BK * gin::BK;
    return (size_t)(2 * Nin * ldk * 2 + 256);
}

// grad_S = W^T grad_I per batch element.  ws: syn_grad_input_ws(N, Nin) bytes, 256-byte aligned.
// Returns 0, a CUDA error code (> 0), or -2 when the tensor maps cannot be built.
int launch_syn_grad_input(long long B, long long N, long long Nin, long long T, const float *W, const float *gI,
                          float *gS, void *ws, int *status, cudaStream_t stream) {
    using namespace gin;
    if (B == 0 || Nin == 0 || T == 0) return 0;
    const long long ldk = (N + BK - 1) / BK * BK;
    uint16_t *hi = static_cast<uint16_t *>(ws);
    uint16_t *lo = hi + Nin * ldk;
    if (N == 0) return (int)cudaMemsetAsync(gS, 0, sizeof(float) * B * Nin * T, stream);
    {
        const long long total = Nin * ldk;
        long long blocks = (total + 255) / 256;
        if (blocks > 65535LL * 8) blocks = 65535LL * 8;
        void *args[] = {const_cast<float **>(&W), &N, &Nin, const_cast<long long *>(&ldk), &hi, &lo};
        const cudaError_t e = cudaLaunchKernel((const void *)wt_split_kernel, dim3((unsigned)blocks), dim3(256), args, 0,
                                               stream);
        if (e != cudaSuccess) return (int)e;
    }
    CUtensorMap mh, ml;
    if (make_wt_map(&mh, hi, Nin, ldk) || make_wt_map(&ml, lo, Nin, ldk)) return -2;
    Args A;
    A.B = B;
    A.N = N;
    A.Nin = Nin;
    A.T = T;
    A.G = gI;
    A.out = gS;
    A.tiles_m = (int)((Nin + BM - 1) / BM);
    A.tiles_t = (int)((T + BN - 1) / BN);
    A.nk = (int)(ldk / BK);
    A.tiles = (long long)A.tiles_m * A.tiles_t * B;
    A.status = status;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        cudaFuncSetAttribute(gin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    }
    const unsigned grid = (unsigned)(A.tiles < sms ? A.tiles : sms);
    void *args[] = {&mh, &ml, &A};
    return (int)cudaLaunchKernel((const void *)gin_kernel, dim3(grid), dim3(THREADS), args, SMEM_BYTES, stream);
}

}  // namespace alif
