// Tensor-map (TMA descriptor) helpers shared by the kernels that stage tiles
// with cp.async.bulk.tensor.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace alif {

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point so
// that the library needs no link against libcuda.  nullptr if unavailable.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP32 currents viewed as n16 rows of 16 floats (64 bytes); one box is box_rows
// such rows (32: 512 consecutive steps of one neuron row; 16: 256 steps), stored
// with the 64-byte swizzle (16-byte chunk q of box row r lands at chunk
// q ^ ((r >> 1) & 3)).  Returns 0, -1 (no encoder) or -2 (rejected).  I must be
// 16-byte aligned.
inline int make_rows16_map(CUtensorMap *map, const float *I, long long n16, unsigned box_rows = 32) {
    auto enc = tensor_map_encoder();
    if (!enc) return -1;
    const cuuint64_t dims[2] = {16, (cuuint64_t)n16};
    const cuuint64_t strides[1] = {64};
    const cuuint32_t box[2] = {16, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(I), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

// FP32 currents as a [rows, T] matrix (row stride T floats); one box is 32 rows x 32 steps
// (4 KB) stored with the 128-byte swizzle (16-byte chunk q of box row y lands at chunk
// q ^ (y & 7)), so that 32 lanes each reading 16 bytes of their own row hit distinct bank
// groups in each quarter warp.  Returns 0, -1 (no encoder) or -2 (rejected: I must be 16-byte
// aligned and T a multiple of 4).
inline int make_rowmajor_map(CUtensorMap *map, const float *I, long long rows, long long T) {
    auto enc = tensor_map_encoder();
    if (!enc) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)T, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)T * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(I), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

// 2-D tiled TMA load global -> shared, completion on the mbarrier at `bar`.
// The inner coordinate c0 times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d_u(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

}  // namespace alif
