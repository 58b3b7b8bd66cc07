// Allocation-free variant of alif_backward().
//
// Some callers cannot allocate device memory at the point where they need the
// backward pass: code running inside a fixed memory budget that was reserved
// up front (an embedded or real-time host loop, a plugin whose host application
// owns the allocator), or code that must not call cudaMalloc/cudaFree because
// those calls synchronise the device and would stall other work.  For them this
// file keeps the backward's scratch -- the per-row partial parameter sums that
// alif_backward() otherwise takes from a caller workspace -- in a fixed-size
// array in the library's own device memory.
//
// The array is a file-scope __device__ object: every GPU that loads the library
// holds ALIF_NOALLOC_MAX_ROWS * 10 floats (2.5 MiB) of it until the process
// exits.  Host code must not pass the array's name to a kernel (on the host it
// is only a stand-in symbol); its device address is looked up once per device
// with cudaGetSymbolAddress, on the first call made while that device is
// current.
#include "common.cuh"

namespace alif {

int launch_alif_backward(long long B, long long N, long long T, const float *I,
                         const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                         const AlifState *ckpt, const float *gS, const float *gV, const float *ga,
                         const float *gfin, float slope, int surrogate, float *gI, float *ginit,
                         float *part, int *status, cudaStream_t stream);
int alif_status_word(int **out);
int alif_record_error(int code, const char *msg);

namespace {

// Per-row partial parameter sums as (hi, lo) pairs: 2 * ALIF_NUM_PARAM_GRADS floats per row.
static __device__ __align__(256) float g_noalloc_scratch[(size_t)ALIF_NOALLOC_MAX_ROWS * 2 * ALIF_NUM_PARAM_GRADS];

constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {nullptr};

int nfail(int code, const char *msg) { return alif_record_error(code, msg); }

// Device address of the scratch array for the current device (looked up once per device).
int scratch_address(float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(ALIF_ECUDA, "alif_backward_noalloc: no current CUDA device");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(ALIF_ECUDA, "alif_backward_noalloc: cudaGetSymbolAddress failed for the scratch array");
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return ALIF_OK;
}

// Batch reduction of the per-row partials in a fixed order (as alif_backward does).
__global__ void noalloc_reduce_kernel(const float *part, float *out, long long B, long long N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    df acc[ALIF_NUM_PARAM_GRADS];
#pragma unroll
    for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) acc[k] = df{0.0f, 0.0f};
    for (long long b = 0; b < B; ++b) {
        const float *q = part + (b * N + i) * (2 * ALIF_NUM_PARAM_GRADS);
#pragma unroll
        for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) acc[k] = df_add(acc[k], df{q[2 * k], q[2 * k + 1]});
    }
#pragma unroll
    for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) out[k * N + i] = acc[k].hi + acc[k].lo;
}

}  // namespace
}  // namespace alif

using namespace alif;

extern "C" int alif_backward_noalloc(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                                     const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                                     const float *grad_spikes, const float *grad_v, const float *grad_a,
                                     const float *grad_final, float slope, float *grad_I, float *grad_init,
                                     float *grad_params, void *stream) {
    if (B < 0 || N < 0 || T < 0) return nfail(ALIF_ESHAPE, "alif_backward_noalloc: negative size");
    const long long rows = (long long)B * N;
    if (rows > ALIF_NOALLOC_MAX_ROWS)
        return nfail(ALIF_ESHAPE,
                     "alif_backward_noalloc: B*N exceeds ALIF_NOALLOC_MAX_ROWS (65536); use alif_backward "
                     "with a workspace");
    if (rows == 0) return ALIF_OK;
    if (T == 0 || !I || !neurons || !spikes || !grad_spikes || !grad_params)
        return nfail(ALIF_EINVAL, "alif_backward_noalloc: needs T > 0 and I, neurons, spikes, grad_spikes, "
                                  "grad_params");
    if (!ckpt && T > ALIF_CKPT_STEPS) return nfail(ALIF_EINVAL, "alif_backward_noalloc: ckpt is required");
    if (!(slope >= 0.0f)) return nfail(ALIF_EINVAL, "alif_backward_noalloc: slope must be >= 0");
    if ((reinterpret_cast<uintptr_t>(neurons) & 15u) != 0)
        return nfail(ALIF_ESHAPE, "alif_backward_noalloc: neurons must be 16-byte aligned");
    float *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    int *status = nullptr;
    if (alif_status_word(&status) != ALIF_OK) status = nullptr;
    // Every row's slot is overwritten by the backward kernel before the
    // reduction reads it, so the array needs no clearing between calls.
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int e = launch_alif_backward(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final,
                                 slope, 0, grad_I, grad_init, scratch, status, st);
    if (e != 0) return nfail(ALIF_ECUDA, "alif_backward_noalloc: kernel launch failed");
    noalloc_reduce_kernel<<<(unsigned)((N + 127) / 128), 128, 0, st>>>(scratch, grad_params, B, N);
    if (cudaGetLastError() != cudaSuccess) return nfail(ALIF_ECUDA, "alif_backward_noalloc: reduction launch failed");
    return ALIF_OK;
}

