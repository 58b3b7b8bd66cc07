// C ABI of the ALIF library: argument validation, FP64 host preparation of
// the per-neuron constants, error reporting, and kernel dispatch.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>


#include "common.cuh"

namespace alif {

size_t alif_forward_fused_ws(long long B, long long Nin, long long T, int cap);
int launch_alif_forward_fused(long long B, long long Nin, long long N, long long T, const float *W,
                              const uint32_t *S, const float *bias, const AlifNeuron *nrn, const AlifState *init,
                              int cap, float *I, uint32_t *spikes, AlifState *ckpt, AlifState *fin, void *ws,
                              unsigned long long *counters, int *status, cudaStream_t stream);
int launch_alif_forward(long long B, long long N, long long T, const float *I,
                        const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                        float *vtr, float *atr, AlifState *ckpt, AlifState *fin,
                        unsigned long long *counters, int *status, cudaStream_t stream);
int launch_alif_forward_recurrent(long long B, long long N, long long T, int TR, const float *Iff, const float *Wt,
                                  const AlifNeuron *nrn, const AlifState *init, float *Iout, uint32_t *spikes,
                                  AlifState *ckpt, AlifState *fin, cudaStream_t stream);
int launch_delay_spikes(long long rows, long long T, long long D, const uint32_t *in, uint32_t *out,
                        cudaStream_t stream);
int launch_alif_forward_seq(long long B, long long N, long long T, const float *I,
                            const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                            float *vtr, float *atr, AlifState *fin, cudaStream_t stream);
int launch_alif_forward_seq_staged(long long B, long long N, long long T, const float *I,
                                   const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                                   float *vtr, float *atr, AlifState *fin, cudaStream_t stream);
int launch_alif_backward_seq(long long B, long long N, long long T, const float *I,
                             const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                             const float *vtr, const float *atr, const float *gS, const float *gV,
                             const float *ga, const float *gfin, float slope, float *gI,
                             float *ginit, float *part, cudaStream_t stream);
int launch_alif_backward(long long B, long long N, long long T, const float *I,
                         const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                         const AlifState *ckpt, const float *gS, const float *gV, const float *ga,
                         const float *gfin, float slope, int surrogate, float *gI, float *ginit,
                         float *part, int *status, cudaStream_t stream);
int launch_alif_backward_attached(long long B, long long N, long long T, const float *I, const AlifNeuron *nrn,
                                  const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                                  const float *gS, const float *gV, const float *ga, const float *gfin,
                                  const float *gfin_s, float slope, int surrogate, float *gI, float *ginit,
                                  float *ginit_s, float *part, cudaStream_t stream);

int launch_split_pad(const float *W, long long N, long long Nin, long long ldw, uint16_t *hi, uint16_t *lo,
                     cudaStream_t stream);
int launch_syn_project(long long B, long long Nin, long long N, long long T, const uint16_t *W_hi,
                       const uint16_t *W_lo, long long ldw, const uint32_t *S, const float *bias, float *I,
                       int *status, cudaStream_t stream);

size_t syn_project_backward_ws(long long B, long long N, long long Nin);
int launch_syn_project_backward(long long B, long long Nin, long long N, long long T, const float *W,
                                const uint32_t *S, const float *gI, float *gW, float *gS, float *gb, void *ws,
                                int *status, cudaStream_t stream);

int launch_readout_forward(long long B, long long K, long long C, long long T, const uint32_t *S, const float *W,
                           const float *bias, const float *w, float w_sum, float *n, float *o, cudaStream_t st);
int launch_readout_backward(long long B, long long K, long long C, long long T, const float *W, const float *w,
                            float w_sum, const float *n, const float *g_o, float *gS, float *gW, float *gb,
                            cudaStream_t st);
int launch_cross_entropy(long long B, long long C, const float *o, const int32_t *y, float *loss, float *g_o,
                         float *row_loss, cudaStream_t st);
int launch_pack_spikes(long long rows, long long T, const float *S, uint32_t *words, cudaStream_t st);
int launch_transpose_weights(const float *W, long long N, long long Nin, float *Wt, cudaStream_t st);
int launch_syn_project_events(long long B, long long Nin, long long N, long long T, const float *Wt,
                              const uint32_t *S, const float *bias, float *I, cudaStream_t st);
int launch_vr_forward(long long rows, long long T, const uint32_t *x, const uint32_t *y, double dec, double scale,
                      long long chunk, float *f_ckpt, float *loss, cudaStream_t st);
int launch_vr_backward(long long rows, long long T, const uint32_t *x, const uint32_t *y, double dec, float gscale,
                       long long t0, long long t1, const float *f_start, float *g_carry, float *grad, long long ldg,
                       cudaStream_t st);

// Device status word and forward counters: module globals, no allocation.
__device__ int g_alif_status = 0;
__device__ unsigned long long g_fwd_counters[4] = {0, 0, 0, 0};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(ALIF_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

struct Symbols {
    int *status = nullptr;
    unsigned long long *counters = nullptr;
};
constexpr int kMaxDevices = 64;
Symbols g_sym[kMaxDevices];

// Device addresses of the module globals for the current device.
int symbols(Symbols **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(ALIF_EUNSUPPORTED, "device ordinal %d", dev);
    Symbols &s = g_sym[dev];
    if (!s.status) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_alif_status);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
        void *q = nullptr;
        e = cudaGetSymbolAddress(&q, g_fwd_counters);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(counters)");
        s.counters = static_cast<unsigned long long *>(q);
        s.status = static_cast<int *>(p);
    }
    *out = &s;
    return ALIF_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_shape(long long B, long long N, long long T) {
    if (B < 0 || N < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size B=%lld N=%lld T=%lld", B, N, T);
    const long long lim = 1LL << 40;
    if (B > lim || N > lim || T > lim) return fail(ALIF_ESHAPE, "size too large");
    if (B && N && (B * N > (1LL << 40) / (T ? T : 1)))
        return fail(ALIF_ESHAPE, "B*N*T = %lld*%lld*%lld exceeds 2^40", B, N, T);
    return ALIF_OK;
}

int launch_status(int rc, const char *what) {
    if (rc != 0) return cuda_fail(static_cast<cudaError_t>(rc), what);
    return ALIF_OK;
}

__global__ void reduce_params_kernel(const float *part, float *out, long long B, long long N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    df acc[ALIF_NUM_PARAM_GRADS];
#pragma unroll
    for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) acc[k] = df{0.0f, 0.0f};
    for (long long b = 0; b < B; ++b) {  // fixed order: deterministic
        const float *q = part + (b * N + i) * (2 * ALIF_NUM_PARAM_GRADS);
#pragma unroll
        for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) acc[k] = df_add(acc[k], df{q[2 * k], q[2 * k + 1]});
    }
#pragma unroll
    for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) out[k * N + i] = acc[k].hi + acc[k].lo;
}

__global__ void copy_state_kernel(const AlifState *init, AlifState *fin, long long rows) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    AlifState s{0.0f, 0.0f, 0};
    if (init) s = init[r];
    fin[r] = s;
}

int reduce_params(const float *part, float *out, long long B, long long N, cudaStream_t st) {
    if (N == 0) return ALIF_OK;
    const int threads = 128;
    // the launch's own status (cudaGetLastError could report an earlier, unrelated failure)
    void *args[] = {&part, &out, &B, &N};
    const cudaError_t e = cudaLaunchKernel((const void *)reduce_params_kernel,
                                           dim3((unsigned)((N + threads - 1) / threads)), dim3(threads), args, 0, st);
    return e == cudaSuccess ? ALIF_OK : cuda_fail(e, "reduce_params_kernel");
}

}  // namespace

// Internal helpers for other translation units of the library.
int alif_status_word(int **out) {
    Symbols *s = nullptr;
    const int rc = symbols(&s);
    if (rc) return rc;
    *out = s->status;
    return ALIF_OK;
}

int alif_record_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace alif

using namespace alif;

extern "C" {

int alif_last_error(char *buf, size_t len) {
    if (buf && len) {
        const size_t n = g_err.size() < len - 1 ? g_err.size() : len - 1;
        memcpy(buf, g_err.data(), n);
        buf[n] = '\0';
    }
    return (int)g_err.size();
}

int alif_device_status(void *stream, int32_t *status_host) {
    if (!status_host) return fail(ALIF_EINVAL, "status_host is NULL");
    Symbols *s = nullptr;
    int rc = symbols(&s);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyAsync(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->status, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "alif_device_status");
    *status_host = v;
    return ALIF_OK;
}

int alif_forward_stats(void *stream, int64_t *out4) {
    if (!out4) return fail(ALIF_EINVAL, "out4 is NULL");
    Symbols *s = nullptr;
    int rc = symbols(&s);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long v[4] = {0, 0, 0, 0}, z[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(v, s->counters, sizeof v, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->counters, z, sizeof z, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "alif_forward_stats");
    for (int k = 0; k < 4; ++k) out4[k] = (int64_t)v[k];
    return ALIF_OK;
}

int alif_tr(double dt_ms, double arp_ms) {
    if (!std::isfinite(dt_ms) || !std::isfinite(arp_ms) || !(dt_ms > 0.0) || !(arp_ms > 0.0))
        return fail(ALIF_EINVAL, "DT and ARP must be finite and > 0 (DT=%g ARP=%g)", dt_ms, arp_ms);
    const double q = arp_ms / dt_ms;
    const double r = std::floor(q + 0.5);
    if (std::fabs(q - r) > 1e-9 * (q > 1.0 ? q : 1.0) || r < 1.0 || r > 1e6)
        return fail(ALIF_ETR, "ARP/DT = %.12g is not an integer >= 1", q);
    return (int)r;
}

int64_t alif_ckpt_count(int64_t T) { return T <= 0 ? 0 : (T + ALIF_CKPT_STEPS - 1) / ALIF_CKPT_STEPS; }

int alif_prepare(int64_t N, const float *tau_mem, const float *tau_adapt, const float *theta0,
                 const float *d_adapt, const float *R, double dt_ms, double arp_ms, AlifNeuron *out) {
    if (N < 0) return fail(ALIF_ESHAPE, "N < 0");
    if (N > 0 && (!tau_mem || !tau_adapt || !theta0 || !d_adapt || !out))
        return fail(ALIF_EINVAL, "NULL parameter array");
    const int tr = alif_tr(dt_ms, arp_ms);
    if (tr < 0) return tr;
    for (int64_t i = 0; i < N; ++i) {
        const double tm = tau_mem[i], ta = tau_adapt[i], th0 = theta0[i], d = d_adapt[i];
        const double r = R ? (double)R[i] : 1.0;
        if (!std::isfinite(tm) || !(tm > 0.0) || !std::isfinite(ta) || !(ta > 0.0))
            return fail(ALIF_EINVAL, "neuron %lld: time constants must be finite and > 0", (long long)i);
        if (!std::isfinite(th0) || !(th0 > 0.0))
            return fail(ALIF_EINVAL, "neuron %lld: theta0 must be > 0", (long long)i);
        if (!std::isfinite(d) || d < 0.0) return fail(ALIF_EINVAL, "neuron %lld: d must be >= 0", (long long)i);
        if (!std::isfinite(r) || r < 0.0) return fail(ALIF_EINVAL, "neuron %lld: R must be >= 0", (long long)i);
        const double beta = std::exp(-dt_ms / tm);  // Eq 2 decay
        const double p = std::exp(-dt_ms / ta);     // Eq 5 decay
        const double c = (1.0 - beta) * r;
        AlifNeuron n;
        memset(&n, 0, sizeof n);
        n.beta_hi = (float)beta;
        n.beta_lo = (float)(beta - (double)n.beta_hi);
        n.p_hi = (float)p;
        n.p_lo = (float)(p - (double)n.p_hi);
        n.c_hi = (float)c;
        n.c_lo = (float)(c - (double)n.c_hi);
        n.theta0 = (float)th0;
        n.d = (float)d;
        n.R = (float)r;
        n.one_minus_beta = (float)(1.0 - beta);
        n.dbeta_dtau = (float)(beta * dt_ms / (tm * tm));
        n.dp_dtau = (float)(p * dt_ms / (ta * ta));
        n.guard = 0.0f;  // reserved: the kernels form their error bounds from the window's own terms
        n.tr = tr;
        n.teff = tr > 2 ? tr : 2;
        out[i] = n;
    }
    return ALIF_OK;
}

int alif_forward(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                 const AlifState *init, uint32_t *spikes, float *v_trace, float *a_trace,
                 AlifState *ckpt, AlifState *final_state, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    const long long rows = (long long)B * N;
    if (rows == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        if (final_state) {
            copy_state_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(init, final_state, rows);
            return launch_status((int)cudaGetLastError(), "copy_state_kernel");
        }
        return ALIF_OK;
    }
    if (!I || !neurons || !spikes) return fail(ALIF_EINVAL, "I, neurons and spikes are required");
    if (!aligned(I, 4) || !aligned(neurons, 16) || !aligned(spikes, 4) || (v_trace && !aligned(v_trace, 4)) ||
        (a_trace && !aligned(a_trace, 4)) || (init && !aligned(init, 4)) || (ckpt && !aligned(ckpt, 4)) ||
        (final_state && !aligned(final_state, 4)))
        return fail(ALIF_ESHAPE, "misaligned pointer (neurons needs 16 bytes, the rest 4)");
    Symbols *s = nullptr;
    rc = symbols(&s);
    if (rc) return rc;
    return launch_status(launch_alif_forward(B, N, T, I, neurons, init, spikes, v_trace, a_trace, ckpt,
                                             final_state, s->counters, s->status, st),
                         "alif_forward launch");
}

size_t alif_forward_fused_workspace_size(int64_t B, int64_t Nin, int64_t T, int32_t max_events_per_word) {
    if (B <= 0 || Nin <= 0 || T <= 0 || max_events_per_word <= 0) return 0;
    return alif_forward_fused_ws(B, Nin, T, max_events_per_word);
}

int alif_forward_fused(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W, const uint32_t *S_in,
                       const float *bias, const AlifNeuron *neurons, const AlifState *init,
                       int32_t max_events_per_word, float *I, uint32_t *spikes, AlifState *ckpt,
                       AlifState *final_state, void *workspace, size_t workspace_bytes, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    if (Nin < 1 || Nin > 1024) return fail(ALIF_EUNSUPPORTED, "alif_forward_fused needs 1 <= Nin <= 1024");
    if (max_events_per_word < 1 || max_events_per_word > 32 * 1024)
        return fail(ALIF_EINVAL, "max_events_per_word must be in [1, 32768]");
    const long long rows = (long long)B * N;
    if (rows == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        if (final_state) {
            copy_state_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(init, final_state, rows);
            return launch_status((int)cudaGetLastError(), "copy_state_kernel");
        }
        return ALIF_OK;
    }
    if (!W || !S_in || !neurons || !I || !spikes) return fail(ALIF_EINVAL, "W, S_in, neurons, I and spikes are required");
    if (!aligned(I, 16) || !aligned(W, 4) || !aligned(S_in, 4) || !aligned(neurons, 16) || !aligned(spikes, 4) ||
        (bias && !aligned(bias, 4)) || (init && !aligned(init, 4)) || (ckpt && !aligned(ckpt, 4)) ||
        (final_state && !aligned(final_state, 4)) || !aligned(workspace, 256))
        return fail(ALIF_ESHAPE, "misaligned pointer (I needs 16 bytes, workspace 256, neurons 16, the rest 4)");
    if (!workspace || workspace_bytes < alif_forward_fused_ws(B, Nin, T, max_events_per_word))
        return fail(ALIF_EWORKSPACE, "workspace too small: need %zu bytes",
                    alif_forward_fused_ws(B, Nin, T, max_events_per_word));
    Symbols *s = nullptr;
    rc = symbols(&s);
    if (rc) return rc;
    return launch_status(launch_alif_forward_fused(B, Nin, N, T, W, S_in, bias, neurons, init, max_events_per_word, I,
                                                   spikes, ckpt, final_state, workspace, s->counters, s->status, st),
                         "alif_forward_fused launch");
}

int alif_forward_recurrent(int64_t B, int64_t N, int64_t T, const float *I_ff, const float *W_rec_t,
                           const AlifNeuron *neurons, double dt_ms, double arp_ms, const AlifState *init,
                           float *I_total, uint32_t *spikes, AlifState *ckpt, AlifState *final_state,
                           void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    const int TR = alif_tr(dt_ms, arp_ms);
    if (TR < 0) return TR;
    if (N > 8192) return fail(ALIF_EUNSUPPORTED, "recurrent layer: N = %lld > 8192", (long long)N);
    if (TR > 1023) return fail(ALIF_EUNSUPPORTED, "recurrent layer: T_R = %d > 1023", TR);
    const long long rows = (long long)B * N;
    if (rows == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        if (final_state) {
            copy_state_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(init, final_state, rows);
            return launch_status((int)cudaGetLastError(), "copy_state_kernel");
        }
        return ALIF_OK;
    }
    if (!I_ff || !W_rec_t || !neurons || !spikes) return fail(ALIF_EINVAL, "I_ff, W_rec_t, neurons and spikes are required");
    if (!aligned(I_ff, 4) || !aligned(W_rec_t, 4) || !aligned(neurons, 16) || !aligned(spikes, 4) ||
        (I_total && !aligned(I_total, 4)) || (init && !aligned(init, 4)) || (ckpt && !aligned(ckpt, 4)) ||
        (final_state && !aligned(final_state, 4)))
        return fail(ALIF_ESHAPE, "misaligned pointer (neurons needs 16 bytes, the rest 4)");
    const int r = launch_alif_forward_recurrent(B, N, T, TR, I_ff, W_rec_t, neurons, init, I_total, spikes, ckpt,
                                                final_state, st);
    if (r < 0) return fail(ALIF_EUNSUPPORTED, "recurrent layer: T_R = %d with N = %lld needs too much shared memory",
                           TR, (long long)N);
    return launch_status(r, "alif_forward_recurrent launch");
}

int alif_delay_spikes(int64_t B, int64_t N, int64_t T, int64_t D, const uint32_t *spikes, uint32_t *delayed,
                      void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    if (D < 0) return fail(ALIF_EINVAL, "delay D = %lld < 0", (long long)D);
    if ((long long)B * N * T == 0) return ALIF_OK;
    if (!spikes || !delayed) return fail(ALIF_EINVAL, "spikes and delayed are required");
    if (spikes == delayed) return fail(ALIF_EINVAL, "the delayed raster must not alias the input");
    return launch_status(launch_delay_spikes((long long)B * N, T, D, spikes, delayed, static_cast<cudaStream_t>(stream)),
                         "alif_delay_spikes launch");
}

int alif_forward_seq(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                     const AlifState *init, uint32_t *spikes, float *v_trace, float *a_trace,
                     AlifState *final_state, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    const long long rows = (long long)B * N;
    if (rows == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        if (final_state) {
            copy_state_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(init, final_state, rows);
            return launch_status((int)cudaGetLastError(), "copy_state_kernel");
        }
        return ALIF_OK;
    }
    if (!I || !neurons || !spikes) return fail(ALIF_EINVAL, "I, neurons and spikes are required");
    if (!aligned(neurons, 16)) return fail(ALIF_ESHAPE, "neurons must be 16-byte aligned");
    return launch_status(
        launch_alif_forward_seq(B, N, T, I, neurons, init, spikes, v_trace, a_trace, final_state, st),
        "alif_forward_seq launch");
}

int alif_forward_seq_staged(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                     const AlifState *init, uint32_t *spikes, float *v_trace, float *a_trace,
                     AlifState *final_state, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    const long long rows = (long long)B * N;
    if (rows == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (T == 0) {
        if (final_state) {
            copy_state_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(init, final_state, rows);
            return launch_status((int)cudaGetLastError(), "copy_state_kernel");
        }
        return ALIF_OK;
    }
    if (!I || !neurons || !spikes) return fail(ALIF_EINVAL, "I, neurons and spikes are required");
    if (!aligned(neurons, 16)) return fail(ALIF_ESHAPE, "neurons must be 16-byte aligned");
    return launch_status(
        launch_alif_forward_seq_staged(B, N, T, I, neurons, init, spikes, v_trace, a_trace, final_state, st),
        "alif_forward_seq_staged launch");
}

size_t alif_backward_workspace_size(int64_t B, int64_t N) {
    if (B <= 0 || N <= 0) return 0;
    return (size_t)B * (size_t)N * 2 * ALIF_NUM_PARAM_GRADS * sizeof(float);
}

// Argument checks every detached/attached block backward shares (the workspace is checked
// by the caller, since alif_backward_noalloc has none).
static int check_backward_args(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                               const uint32_t *spikes, const float *grad_spikes, float *grad_params, float slope) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    if (!std::isfinite(slope) || slope < 0.0f) return fail(ALIF_EINVAL, "slope must be finite and >= 0");
    if ((long long)B * N == 0) return ALIF_OK;
    if (!neurons || !grad_params) return fail(ALIF_EINVAL, "neurons and grad_params are required");
    if (T > 0 && (!I || !spikes || !grad_spikes)) return fail(ALIF_EINVAL, "I, spikes and grad_spikes are required");
    if (!aligned(neurons, 16)) return fail(ALIF_ESHAPE, "neurons must be 16-byte aligned");
    return ALIF_OK;
}

static int check_backward_common(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                                 const uint32_t *spikes, const float *grad_spikes, float *grad_params,
                                 void *workspace, size_t workspace_bytes, float slope) {
    int rc = check_backward_args(B, N, T, I, neurons, spikes, grad_spikes, grad_params, slope);
    if (rc) return rc;
    if ((long long)B * N == 0) return ALIF_OK;
    if (workspace_bytes < alif_backward_workspace_size(B, N) || !workspace)
        return fail(ALIF_EWORKSPACE, "workspace too small: need %zu bytes", alif_backward_workspace_size(B, N));
    return ALIF_OK;
}

int alif_backward_seq(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                      const AlifState *init, const uint32_t *spikes, const float *v_trace,
                      const float *a_trace, const float *grad_spikes, const float *grad_v,
                      const float *grad_a, const float *grad_final, float slope, float *grad_I,
                      float *grad_init, float *grad_params, void *workspace, size_t workspace_bytes,
                      void *stream) {
    int rc = check_backward_common(B, N, T, I, neurons, spikes, grad_spikes, grad_params, workspace,
                                   workspace_bytes, slope);
    if (rc) return rc;
    if ((long long)B * N == 0) return ALIF_OK;
    if (T > 0 && (!v_trace || !a_trace)) return fail(ALIF_EINVAL, "v_trace and a_trace are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *part = static_cast<float *>(workspace);
    rc = launch_status(launch_alif_backward_seq(B, N, T, I, neurons, init, spikes, v_trace, a_trace,
                                                grad_spikes, grad_v, grad_a, grad_final, slope, grad_I,
                                                grad_init, part, st),
                       "alif_backward_seq launch");
    if (rc) return rc;
    return reduce_params(part, grad_params, B, N, st);
}

int alif_backward(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                  const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                  const float *grad_spikes, const float *grad_v, const float *grad_a,
                  const float *grad_final, float slope, float *grad_I, float *grad_init,
                  float *grad_params, void *workspace, size_t workspace_bytes, void *stream) {
    return alif_backward_surrogate(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a,
                                   grad_final, ALIF_SG_FAST_SIGMOID, slope, grad_I, grad_init, grad_params,
                                   workspace, workspace_bytes, stream);
}

// Pointer checks of the block backward, made before any CUDA call: the checkpoints are
// required past the first 256 steps, and every array must be 4-byte aligned.
static int check_backward_ptrs(int64_t T, const float *I, const AlifState *init, const uint32_t *spikes,
                               const AlifState *ckpt, const float *grad_spikes, const float *grad_v,
                               const float *grad_a, const float *grad_final, const float *grad_I,
                               const float *grad_init, const float *grad_params) {
    if (T > 0 && !ckpt && T > ALIF_CKPT_STEPS)
        return fail(ALIF_EINVAL, "ckpt is required when T > %d", ALIF_CKPT_STEPS);
    if ((I && !aligned(I, 4)) || (grad_spikes && !aligned(grad_spikes, 4)) || (grad_v && !aligned(grad_v, 4)) ||
        (grad_a && !aligned(grad_a, 4)) || (grad_I && !aligned(grad_I, 4)) || (ckpt && !aligned(ckpt, 4)) ||
        (init && !aligned(init, 4)) || (spikes && !aligned(spikes, 4)) || (grad_final && !aligned(grad_final, 4)) ||
        (grad_init && !aligned(grad_init, 4)) || !aligned(grad_params, 4))
        return fail(ALIF_ESHAPE, "misaligned pointer (arrays need 4-byte alignment)");
    return ALIF_OK;
}

// The block backward after argument checks: T = 0 handling, pointer alignment, the kernel
// and the batch reduction of the per-row partials in `part` (B*N*10 floats).
static int backward_run(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                        const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                        const float *grad_spikes, const float *grad_v, const float *grad_a,
                        const float *grad_final, int surrogate, float slope, bool attached,
                        const float *grad_final_spike, float *grad_I, float *grad_init, float *grad_init_spike,
                        float *grad_params, float *part, cudaStream_t st) {
    if (T == 0) {
        cudaError_t e = cudaMemsetAsync(grad_params, 0, sizeof(float) * ALIF_NUM_PARAM_GRADS * N, st);
        if (e == cudaSuccess && grad_init) {
            // dL/d(init) = dL/d(final) when no step is taken
            e = grad_final ? cudaMemcpyAsync(grad_init, grad_final, sizeof(float) * 2 * B * N,
                                             cudaMemcpyDeviceToDevice, st)
                           : cudaMemsetAsync(grad_init, 0, sizeof(float) * 2 * B * N, st);
        }
        if (e == cudaSuccess && grad_init_spike)
            e = grad_final_spike ? cudaMemcpyAsync(grad_init_spike, grad_final_spike, sizeof(float) * B * N,
                                                   cudaMemcpyDeviceToDevice, st)
                                 : cudaMemsetAsync(grad_init_spike, 0, sizeof(float) * B * N, st);
        return e == cudaSuccess ? ALIF_OK : cuda_fail(e, "alif_backward (T = 0)");
    }
    Symbols *s = nullptr;
    int rc = symbols(&s);
    if (rc) return rc;
    if (attached)
        rc = launch_status(launch_alif_backward_attached(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes,
                                                         grad_v, grad_a, grad_final, grad_final_spike, slope,
                                                         surrogate, grad_I, grad_init, grad_init_spike, part, st),
                           "alif_backward_attached launch");
    else
        rc = launch_status(launch_alif_backward(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v,
                                                grad_a, grad_final, slope, surrogate, grad_I, grad_init, part,
                                                s->status, st),
                           "alif_backward launch");
    if (rc) return rc;
    return reduce_params(part, grad_params, B, N, st);
}

static int backward_impl(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                         const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                         const float *grad_spikes, const float *grad_v, const float *grad_a,
                         const float *grad_final, int surrogate, float slope, bool attached,
                         const float *grad_final_spike, float *grad_I, float *grad_init, float *grad_init_spike,
                         float *grad_params, void *workspace, size_t workspace_bytes, void *stream) {
    if (surrogate < ALIF_SG_FAST_SIGMOID || surrogate > ALIF_SG_BOXCAR)
        return fail(ALIF_EINVAL, "unknown surrogate %d", surrogate);
    int rc = check_backward_common(B, N, T, I, neurons, spikes, grad_spikes, grad_params, workspace,
                                   workspace_bytes, slope);
    if (rc) return rc;
    if ((long long)B * N == 0) return ALIF_OK;
    rc = check_backward_ptrs(T, I, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final, grad_I, grad_init,
                             grad_params);
    if (rc) return rc;
    return backward_run(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final, surrogate,
                        slope, attached, grad_final_spike, grad_I, grad_init, grad_init_spike, grad_params,
                        static_cast<float *>(workspace), static_cast<cudaStream_t>(stream));
}

extern "C++" {
namespace alif {
// The detached fast-sigmoid backward with the per-row partials in scratch that `scratch`
// provides (B*N*10 floats), asked for only once the arguments have passed the same checks
// as alif_backward() (without the workspace check).  Used by the allocation-free entry point.
int alif_backward_into(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                       const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                       const float *grad_spikes, const float *grad_v, const float *grad_a,
                       const float *grad_final, float slope, float *grad_I, float *grad_init,
                       float *grad_params, int (*scratch)(float **), cudaStream_t st) {
    int rc = check_backward_args(B, N, T, I, neurons, spikes, grad_spikes, grad_params, slope);
    if (rc) return rc;
    if ((long long)B * N == 0) return ALIF_OK;
    rc = check_backward_ptrs(T, I, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final, grad_I, grad_init,
                             grad_params);
    if (rc) return rc;
    float *part = nullptr;
    rc = scratch(&part);
    if (rc) return rc;
    return backward_run(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final,
                        ALIF_SG_FAST_SIGMOID, slope, false, nullptr, grad_I, grad_init, nullptr, grad_params, part,
                        st);
}
}  // namespace alif
}  // extern "C++"

int alif_backward_surrogate(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                            const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                            const float *grad_spikes, const float *grad_v, const float *grad_a,
                            const float *grad_final, int surrogate, float slope, float *grad_I,
                            float *grad_init, float *grad_params, void *workspace, size_t workspace_bytes,
                            void *stream) {
    return backward_impl(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final,
                         surrogate, slope, false, nullptr, grad_I, grad_init, nullptr, grad_params, workspace,
                         workspace_bytes, stream);
}

int alif_backward_attached(int64_t B, int64_t N, int64_t T, const float *I, const AlifNeuron *neurons,
                           const AlifState *init, const uint32_t *spikes, const AlifState *ckpt,
                           const float *grad_spikes, const float *grad_v, const float *grad_a,
                           const float *grad_final, const float *grad_final_spike, int surrogate, float slope,
                           float *grad_I, float *grad_init, float *grad_init_spike, float *grad_params,
                           void *workspace, size_t workspace_bytes, void *stream) {
    return backward_impl(B, N, T, I, neurons, init, spikes, ckpt, grad_spikes, grad_v, grad_a, grad_final,
                         surrogate, slope, true, grad_final_spike, grad_I, grad_init, grad_init_spike,
                         grad_params, workspace, workspace_bytes, stream);
}

int syn_split_bf16(const float *W, int64_t N, int64_t Nin, int64_t ldw, uint16_t *W_hi, uint16_t *W_lo,
                   void *stream) {
    if (N < 0 || Nin < 0 || ldw < Nin) return fail(ALIF_ESHAPE, "need N, Nin >= 0 and ldw >= Nin");
    if (N == 0 || ldw == 0) return ALIF_OK;
    if ((Nin > 0 && !W) || !W_hi || !W_lo) return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_split_pad(W, N, Nin, ldw, W_hi, W_lo, static_cast<cudaStream_t>(stream)),
                         "split_pad_kernel");
}

__global__ void bias_fill_kernel(const float *bias, float *I, long long N, long long T, long long total) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x)
        I[k] = bias ? bias[(k / T) % N] : 0.0f;
}

int syn_project(int64_t B, int64_t Nin, int64_t N, int64_t T, const uint16_t *W_hi, const uint16_t *W_lo,
                int64_t ldw, const uint32_t *S_in, const float *bias, float *I, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    if (Nin < 0 || ldw < Nin || ldw % ALIF_PROJ_K_ALIGN != 0)
        return fail(ALIF_ESHAPE, "ldw must be >= Nin and a multiple of %d", ALIF_PROJ_K_ALIGN);
    if ((long long)B * N * T == 0) return ALIF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!I) return fail(ALIF_EINVAL, "I is NULL");
    if (!aligned(I, 4)) return fail(ALIF_ESHAPE, "I must be 4-byte aligned");
    if (Nin == 0) {
        const long long total = (long long)B * N * T;
        long long blocks = (total + 255) / 256;
        if (blocks > 65535LL * 8) blocks = 65535LL * 8;
        bias_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(bias, I, N, T, total);
        return launch_status((int)cudaGetLastError(), "bias_fill_kernel");
    }
    if (!W_hi || !W_lo || !S_in) return fail(ALIF_EINVAL, "W_hi, W_lo and S_in are required");
    if (!aligned(W_hi, 16) || !aligned(W_lo, 16) || !aligned(S_in, 4))
        return fail(ALIF_ESHAPE, "W_hi/W_lo must be 16-byte aligned");
    Symbols *s = nullptr;
    rc = symbols(&s);
    if (rc) return rc;
    const int r = launch_syn_project(B, Nin, N, T, W_hi, W_lo, ldw, S_in, bias, I, s->status, st);
    if (r < 0) return fail(ALIF_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable or rejected the weights");
    return launch_status(r, "syn_project launch");
}

size_t syn_project_backward_workspace_size(int64_t B, int64_t N, int64_t Nin) {
    if (B <= 0 || N <= 0 || Nin < 0) return 0;
    return syn_project_backward_ws(B, N, Nin);
}

int syn_project_backward(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W, const uint32_t *S_in,
                         const float *grad_I, float *grad_W, float *grad_Sin, float *grad_bias, void *workspace,
                         size_t workspace_bytes, void *stream) {
    int rc = check_shape(B, N, T);
    if (rc) return rc;
    if (Nin < 0) return fail(ALIF_ESHAPE, "Nin < 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool zero_work = (long long)B * N * T == 0 || Nin == 0;
    if (zero_work) {  // empty sums
        cudaError_t e = cudaSuccess;
        if (grad_W && N * Nin) e = cudaMemsetAsync(grad_W, 0, sizeof(float) * N * Nin, st);
        if (e == cudaSuccess && grad_bias && N) e = cudaMemsetAsync(grad_bias, 0, sizeof(float) * N, st);
        if (e == cudaSuccess && grad_Sin && B * Nin * T) e = cudaMemsetAsync(grad_Sin, 0, sizeof(float) * B * Nin * T, st);
        return e == cudaSuccess ? ALIF_OK : cuda_fail(e, "syn_project_backward (empty)");
    }
    if (!grad_I) return fail(ALIF_EINVAL, "grad_I is required");
    if ((grad_W || grad_bias) && !S_in) return fail(ALIF_EINVAL, "S_in is required for grad_W / grad_bias");
    if (grad_Sin && !W) return fail(ALIF_EINVAL, "W is required for grad_Sin");
    if ((grad_W || grad_bias || grad_Sin) && (!workspace || workspace_bytes < syn_project_backward_ws(B, N, Nin)))
        return fail(ALIF_EWORKSPACE, "workspace too small: need %zu bytes", syn_project_backward_ws(B, N, Nin));
    if (!aligned(grad_I, 4) || (W && !aligned(W, 4)) || (grad_Sin && !aligned(grad_Sin, 4)) ||
        (S_in && !aligned(S_in, 4)) || !aligned(workspace, 256))
        return fail(ALIF_ESHAPE, "misaligned pointer (workspace needs 256 bytes, the rest 4)");
    Symbols *sy = nullptr;
    rc = symbols(&sy);
    if (rc) return rc;
    const int r = launch_syn_project_backward(B, Nin, N, T, W, S_in, grad_I, grad_W, grad_Sin, grad_bias, workspace,
                                              sy->status, st);
    if (r < 0) return fail(ALIF_EUNSUPPORTED, "syn_project_backward: the driver cannot encode the tensor maps");
    return launch_status(r, "syn_project_backward launch");
}

// One warp per (row, 32-word chunk): the chunk's words are read coalesced, then each of the
// 32 words is broadcast and its bits written as 32 consecutive floats (128 bytes per store).
__global__ void unpack_spikes_kernel(const uint32_t *spikes, float *out, long long rows, long long T, long long nw) {
    const long long nch = (nw + 31) / 32;  // 1024-step chunks per row
    const long long total = rows * nch;
    const int lane = threadIdx.x & 31;
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < total; q += wstride) {
        const long long r = q / nch, c = q - r * nch;
        const long long w = c * 32 + lane;
        const uint32_t mine = w < nw ? spikes[r * nw + w] : 0u;
        float *orow = out + r * T;
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const uint32_t wk = __shfl_sync(0xffffffffu, mine, k);
            const long long t = (c * 32 + k) * 32 + lane;
            if (t < T) orow[t] = (float)((wk >> lane) & 1u);
        }
    }
}

int alif_unpack_spikes(int64_t rows, int64_t T, const uint32_t *spikes, float *out, void *stream) {
    if (rows < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (rows * T == 0) return ALIF_OK;
    if (!spikes || !out) return fail(ALIF_EINVAL, "NULL pointer");
    const long long nw = (T + 31) / 32;
    long long blocks = (rows * ((nw + 31) / 32) + 7) / 8;  // 8 warps per block, one (row, chunk) each
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    unpack_spikes_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(spikes, out, rows, T, nw);
    return launch_status((int)cudaGetLastError(), "unpack_spikes_kernel");
}

int alif_vanrossum_forward(int64_t rows, int64_t T, const uint32_t *x, const uint32_t *y, double dt_ms,
                           double tau_ms, int64_t chunk, float *f_ckpt, float *loss, void *stream) {
    if (rows < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (!(dt_ms > 0.0) || !(tau_ms > 0.0) || !std::isfinite(dt_ms) || !std::isfinite(tau_ms))
        return fail(ALIF_EINVAL, "DT and tau_R must be finite and > 0");
    if (chunk <= 0 || chunk % 256 != 0) return fail(ALIF_EINVAL, "chunk must be a positive multiple of 256");
    if (rows == 0 || T == 0) return ALIF_OK;
    if (!x || !y) return fail(ALIF_EINVAL, "x and y are required");
    return launch_status(launch_vr_forward(rows, T, x, y, std::exp(-dt_ms / tau_ms), dt_ms / tau_ms, chunk, f_ckpt,
                                           loss, static_cast<cudaStream_t>(stream)),
                         "vr_forward_kernel");
}

int alif_vanrossum_backward(int64_t rows, int64_t T, const uint32_t *x, const uint32_t *y, double dt_ms,
                            double tau_ms, int64_t t0, int64_t t1, const float *f_start, float *g_carry, float *grad,
                            void *stream) {
    if (rows < 0 || T < 0 || t0 < 0 || t1 > T || t1 < t0 || t0 % 256 != 0)
        return fail(ALIF_ESHAPE, "need 0 <= t0 <= t1 <= T with t0 a multiple of 256");
    if (!(dt_ms > 0.0) || !(tau_ms > 0.0)) return fail(ALIF_EINVAL, "DT and tau_R must be > 0");
    if (rows == 0 || t1 == t0) return ALIF_OK;
    if (!x || !y || !f_start || !g_carry || !grad) return fail(ALIF_EINVAL, "NULL pointer");
    // the kernel keeps one float per 256-step window and warp in shared memory (<= 32 KB)
    if ((t1 - t0) > (1LL << 19)) return fail(ALIF_EUNSUPPORTED, "chunk longer than 2^19 steps");
    return launch_status(launch_vr_backward(rows, T, x, y, std::exp(-dt_ms / tau_ms), (float)(2.0 * dt_ms / tau_ms),
                                            t0, t1, f_start, g_carry, grad, t1 - t0,
                                            static_cast<cudaStream_t>(stream)),
                         "vr_backward_kernel");
}

int alif_readout_weights(int64_t T, double dt_ms, double tau_ms, float *w_t, double *w_sum) {
    if (T < 0) return fail(ALIF_ESHAPE, "T < 0");
    if (!std::isfinite(dt_ms) || !std::isfinite(tau_ms) || !(dt_ms > 0.0) || !(tau_ms > 0.0))
        return fail(ALIF_EINVAL, "DT and tau must be finite and > 0");
    if (T > 0 && (!w_t || !w_sum)) return fail(ALIF_EINVAL, "w_t and w_sum are required");
    const double beta = std::exp(-dt_ms / tau_ms);
    double sum = 0.0, bp = 1.0;  // beta^(T - t), built from t = T - 1 down
    for (int64_t t = T - 1; t >= 0; --t) {
        bp *= beta;
        const double w = 1.0 - bp;
        w_t[t] = (float)w;
        sum += w;
    }
    if (w_sum) *w_sum = sum;
    return ALIF_OK;
}

int alif_readout_forward(int64_t B, int64_t K, int64_t C, int64_t T, const uint32_t *spikes, const float *W,
                         const float *bias, const float *w_t, float w_sum, float *counts, float *out, void *stream) {
    if (B < 0 || K < 0 || C < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (B == 0 || C == 0) return ALIF_OK;
    if (!W || !counts || !out || (K > 0 && T > 0 && (!spikes || !w_t)))
        return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_readout_forward(B, K, C, T, spikes, W, bias, w_t, w_sum, counts, out,
                                                static_cast<cudaStream_t>(stream)),
                         "readout forward");
}

int alif_readout_backward(int64_t B, int64_t K, int64_t C, int64_t T, const float *W, const float *w_t,
                          float w_sum, const float *counts, const float *grad_out, float *grad_spikes,
                          float *grad_W, float *grad_bias, void *stream) {
    if (B < 0 || K < 0 || C < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (B == 0) return ALIF_OK;
    if (!grad_out || (grad_spikes && (!W || !w_t)) || (grad_W && !counts))
        return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_readout_backward(B, K, C, T, W, w_t, w_sum, counts, grad_out, grad_spikes, grad_W,
                                                 grad_bias, static_cast<cudaStream_t>(stream)),
                         "readout backward");
}

int alif_cross_entropy(int64_t B, int64_t C, const float *logits, const int32_t *labels, float *loss,
                       float *grad_logits, float *workspace, void *stream) {
    if (B <= 0 || C <= 0) return fail(ALIF_ESHAPE, "need B >= 1 and C >= 1");
    if (!logits || !labels || !loss || !workspace) return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_cross_entropy(B, C, logits, labels, loss, grad_logits, workspace,
                                              static_cast<cudaStream_t>(stream)),
                         "cross entropy");
}

int alif_pack_spikes(int64_t rows, int64_t T, const float *S, uint32_t *spikes, void *stream) {
    if (rows < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (rows == 0 || T == 0) return ALIF_OK;
    if (!S || !spikes) return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_pack_spikes(rows, T, S, spikes, static_cast<cudaStream_t>(stream)), "pack spikes");
}

int syn_transpose_weights(const float *W, int64_t N, int64_t Nin, float *W_t, void *stream) {
    if (N < 0 || Nin < 0) return fail(ALIF_ESHAPE, "negative size");
    if (N == 0 || Nin == 0) return ALIF_OK;
    if (!W || !W_t) return fail(ALIF_EINVAL, "NULL pointer");
    return launch_status(launch_transpose_weights(W, N, Nin, W_t, static_cast<cudaStream_t>(stream)),
                         "transpose_kernel");
}

int syn_project_events(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W_t, const uint32_t *S_in,
                       const float *bias, float *I, void *stream) {
    if (B < 0 || Nin < 0 || N < 0 || T < 0) return fail(ALIF_ESHAPE, "negative size");
    if (B == 0 || N == 0 || T == 0) return ALIF_OK;
    if (Nin == 0) {  // no inputs: I = bias
        return launch_status(launch_syn_project_events(B, 0, N, T, W_t, S_in, bias, I,
                                                       static_cast<cudaStream_t>(stream)),
                             "syn_project_events");
    }
    if (!W_t || !S_in || !I) return fail(ALIF_EINVAL, "NULL pointer");
    if (((Nin + 1023) / 1024) * 1024 * N >= (1LL << 31))
        return fail(ALIF_EUNSUPPORTED, "syn_project_events needs ceil(Nin/1024)*1024*N < 2^31");
    return launch_status(launch_syn_project_events(B, Nin, N, T, W_t, S_in, bias, I, static_cast<cudaStream_t>(stream)),
                         "syn_project_events");
}

}  // extern "C"
