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
#include <atomic>

#include "common.cuh"

namespace alif {

int alif_backward_into(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                       const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                       const float *grad_spikes, const float *grad_v, const float *grad_a,
                       const float *grad_final, float slope, float *grad_I, float *grad_init,
                       float *grad_params, int (*scratch)(float **), cudaStream_t st);
int alif_record_error(int code, const char *msg);

namespace {

// Per-row partial parameter sums as (hi, lo) pairs: 2 * ALIF_NUM_PARAM_GRADS floats per row.
static __device__ __align__(256) float g_noalloc_scratch[(size_t)ALIF_NOALLOC_MAX_ROWS * 2 * ALIF_NUM_PARAM_GRADS];

// Device address of the array per device ordinal.  Two host threads making their first call
// on the same device at the same time both look it up and store the same value; the atomic
// makes that store well defined.
constexpr int kMaxDevices = 64;
std::atomic<float *> g_scratch_addr[kMaxDevices];

int nfail(int code, const char *msg) { return alif_record_error(code, msg); }

// Device address of the scratch array for the current device (looked up once per device).
int scratch_address(float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(ALIF_ECUDA, "alif_backward_noalloc: no current CUDA device");
    float *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(ALIF_ECUDA, "alif_backward_noalloc: cudaGetSymbolAddress failed for the scratch array");
        addr = static_cast<float *>(p);
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    *out = addr;
    return ALIF_OK;
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
    if (N > 0 && B > ALIF_NOALLOC_MAX_ROWS / N)
        return nfail(ALIF_ESHAPE,
                     "alif_backward_noalloc: B*N exceeds ALIF_NOALLOC_MAX_ROWS (65536); use alif_backward "
                     "with a workspace");
    // Every check alif_backward() makes runs before the scratch address is looked up, so a
    // rejected call makes no CUDA call.  Every row's slot is overwritten by the backward
    // kernel before the reduction reads it, so the array needs no clearing between calls.
    return alif_backward_into(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final,
                              slope, grad_I, grad_init, grad_params, scratch_address, static_cast<cudaStream_t>(stream));
}
