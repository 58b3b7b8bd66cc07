// Leaky readout and cross-entropy of the classification network
// (Supplementary, "Classification"), and float -> bit packing of spike trains.
//
// The readout is an integrator without spike or reset whose membrane is
// summed over time:
//     V_o[t] = beta_o V_o[t-1] + (1 - beta_o) I_o[t],   o[b,c] = sum_t V_o[t],
//     I_o[b,c,t] = bias_c + sum_k W[c,k] S[b,k,t].
// Summing the impulse response over the remaining steps,
//     o[b,c] = sum_k W[c,k] n[b,k] + bias_c sum_t w_t,
//     n[b,k] = sum_t w_t S[b,k,t],   w_t = 1 - beta_o^(T-t),
// so the forward is a weighted count of each input row's spikes (event
// driven: only set bits are visited) followed by a [B,K] x [K,C] product.
// Backward: dL/dS[b,k,t] = w_t h[b,k] with h[b,k] = sum_c W[c,k] g_o[b,c];
// dL/dW[c,k] = sum_b g_o[b,c] n[b,k]; dL/dbias_c = sum_b g_o[b,c] sum_t w_t.
// All sums run in a fixed order (deterministic).
#include "common.cuh"

namespace alif {
namespace ro {

// n[r] = sum_t w[t] S[r,t]: one warp per row, lanes stride over the words.
__global__ void count_kernel(long long rows, long long T, long long nwords, const uint32_t *__restrict__ S,
                             const float *__restrict__ w, float *n) {
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float acc = 0.0f;
    for (long long q = lane; q < nwords; q += 32) {
        uint32_t word = __ldg(S + r * nwords + q);
        if (q == nwords - 1 && (T & 31)) word &= (1u << (T & 31)) - 1u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            acc += __ldg(w + q * 32 + b);
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) n[r] = acc;
}

// o[b,c] = sum_k W[c,k] n[b,k] + bias_c w_sum: one thread per (b, c).
__global__ void out_kernel(long long B, long long K, long long C, const float *__restrict__ W,
                           const float *__restrict__ bias, float w_sum, const float *__restrict__ n, float *o) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * C) return;
    const long long b = e / C, c = e % C;
    float acc = 0.0f;
    for (long long k = 0; k < K; ++k) acc = fmaf(W[c * K + k], n[b * K + k], acc);
    if (bias) acc = fmaf(bias[c], w_sum, acc);
    o[e] = acc;
}

// dL/dS[r, t] = w[t] h[r], h[b,k] = sum_c W[c,k] g_o[b,c]: one warp per row (b, k).
__global__ void grad_spikes_kernel(long long B, long long K, long long C, long long T, const float *__restrict__ W,
                                   const float *__restrict__ g_o, const float *__restrict__ w, float *gS) {
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= B * K) return;
    const long long b = r / K, k = r % K;
    float h = 0.0f;
    for (long long c = 0; c < C; ++c) h = fmaf(W[c * K + k], g_o[b * C + c], h);
    float *out = gS + r * T;
    if ((T & 3) == 0 && ((reinterpret_cast<uintptr_t>(gS) & 15u) == 0) &&
        ((reinterpret_cast<uintptr_t>(w) & 15u) == 0)) {
        for (long long t = 4LL * lane; t < T; t += 128) {
            const float4 wv = *reinterpret_cast<const float4 *>(w + t);
            *reinterpret_cast<float4 *>(out + t) = make_float4(h * wv.x, h * wv.y, h * wv.z, h * wv.w);
        }
    } else {
        for (long long t = lane; t < T; t += 32) out[t] = h * w[t];
    }
}

// dL/dW[c,k] = sum_b g_o[b,c] n[b,k]; dL/dbias_c = sum_b g_o[b,c] w_sum.
__global__ void grad_w_kernel(long long B, long long K, long long C, const float *__restrict__ g_o,
                              const float *__restrict__ n, float w_sum, float *gW, float *gb) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < C * K && gW) {
        const long long c = e / K, k = e % K;
        float acc = 0.0f;
        for (long long b = 0; b < B; ++b) acc = fmaf(g_o[b * C + c], n[b * K + k], acc);
        gW[e] = acc;
    }
    if (e < C && gb) {
        float acc = 0.0f;
        for (long long b = 0; b < B; ++b) acc += g_o[b * C + e];
        gb[e] = acc * w_sum;
    }
}

// Mean softmax cross-entropy: one block; thread b owns row b (and b + blockDim ...).
__global__ void ce_kernel(long long B, long long C, const float *__restrict__ o, const int32_t *__restrict__ y,
                          float *loss, float *g_o, float *row_loss) {
    for (long long b = threadIdx.x; b < B; b += blockDim.x) {
        const float *ob = o + b * C;
        float m = ob[0];
        for (long long c = 1; c < C; ++c) m = fmaxf(m, ob[c]);
        float s = 0.0f;
        for (long long c = 0; c < C; ++c) s += expf(ob[c] - m);
        const int lab = y[b];
        const bool ok = lab >= 0 && lab < C;  // an invalid label gives a NaN loss, no access
        row_loss[b] = ok ? -(ob[lab] - m - logf(s)) : __int_as_float(0x7fc00000);
        if (g_o) {
            const float inv = 1.0f / ((float)B * s);
            for (long long c = 0; c < C; ++c)
                g_o[b * C + c] = expf(ob[c] - m) * inv - (c == lab ? 1.0f / (float)B : 0.0f);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (long long b = 0; b < B; ++b) acc += (double)row_loss[b];
        *loss = (float)(acc / (double)B);
    }
}

// words[r, q] bit i = (S[r, 32 q + i] != 0): one warp per row, ballot per 32 steps.
__global__ void pack_kernel(long long rows, long long T, long long nwords, const float *__restrict__ S,
                            uint32_t *words) {
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    for (long long q = 0; q < nwords; ++q) {
        const long long t = q * 32 + lane;
        const bool on = t < T && S[r * T + t] != 0.0f;
        const uint32_t word = __ballot_sync(FULL, on);
        if (lane == 0) words[r * nwords + q] = word;
    }
}

}  // namespace ro

int launch_readout_forward(long long B, long long K, long long C, long long T, const uint32_t *S, const float *W,
                           const float *bias, const float *w, float w_sum, float *n, float *o, cudaStream_t st) {
    const long long rows = B * K, nwords = (T + 31) / 32;
    if (rows > 0) {
        ro::count_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(rows, T, nwords, S, w, n);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    if (B * C > 0) {
        ro::out_kernel<<<(unsigned)((B * C + 127) / 128), 128, 0, st>>>(B, K, C, W, bias, w_sum, n, o);
        return (int)cudaGetLastError();
    }
    return 0;
}

int launch_readout_backward(long long B, long long K, long long C, long long T, const float *W, const float *w,
                            float w_sum, const float *n, const float *g_o, float *gS, float *gW, float *gb,
                            cudaStream_t st) {
    if (gS && B * K > 0 && T > 0) {
        ro::grad_spikes_kernel<<<(unsigned)((B * K + 7) / 8), 256, 0, st>>>(B, K, C, T, W, g_o, w, gS);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    const long long m = C * K > C ? C * K : C;
    if ((gW || gb) && m > 0) {
        ro::grad_w_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(B, K, C, g_o, n, w_sum, gW, gb);
        return (int)cudaGetLastError();
    }
    return 0;
}

int launch_cross_entropy(long long B, long long C, const float *o, const int32_t *y, float *loss, float *g_o,
                         float *row_loss, cudaStream_t st) {
    ro::ce_kernel<<<1, 256, 0, st>>>(B, C, o, y, loss, g_o, row_loss);
    return (int)cudaGetLastError();
}

int launch_pack_spikes(long long rows, long long T, const float *S, uint32_t *words, cudaStream_t st) {
    if (rows <= 0 || T <= 0) return 0;
    ro::pack_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(rows, T, (T + 31) / 32, S, words);
    return (int)cudaGetLastError();
}

}  // namespace alif
