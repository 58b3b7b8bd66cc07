// van Rossum distance between spike trains (Supplementary, "Neural fits"),
// the loss of the neuron-fitting requests, and its gradient with respect to the
// model's spike train.  Discretised with the exponential kernel
// k[t] = exp(-t DT / tau_R):
//     f[t] = decay f[t-1] + (x[t] - y[t]),      decay = exp(-DT / tau_R)
//     L    = (DT / tau_R) sum_t f[t]^2           (the squared distance D_R^2)
//     dL/dx[t] = (2 DT / tau_R) g[t],  g[t] = f[t] + decay g[t+1]
// One warp per row, 256-step windows (lane L holds steps 8L..8L+7), decayed
// warp scans in both directions.  The forward saves f entering every chunk of
// `chunk` steps so that the gradient can be produced chunk by chunk, last chunk
// first, alongside a chunked backward of the neuron model.
#include "common.cuh"

namespace alif {
namespace vr {

constexpr int E = 8, WIN = 256, WARPS = 4;

__device__ __forceinline__ void scan_fwd(float (&v)[E], float dec, const float (&Bl)[5], const float (&dk)[E],
                                         int lane) {
#pragma unroll
    for (int k = 1; k < E; ++k) v[k] = fmaf(dec, v[k - 1], v[k]);
    float tot = v[E - 1];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const float up = __shfl_up_sync(FULL, tot, 1 << l);
        if (lane >= (1 << l)) tot = fmaf(Bl[l], up, tot);
    }
    float P = __shfl_up_sync(FULL, tot, 1);
    if (lane == 0) P = 0.0f;
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = fmaf(dk[k], P, v[k]);
}

__device__ __forceinline__ void scan_rev(float (&v)[E], float dec, const float (&Bl)[5], const float (&dk)[E],
                                         int lane) {
#pragma unroll
    for (int k = E - 2; k >= 0; --k) v[k] = fmaf(dec, v[k + 1], v[k]);
    float tot = v[0];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        const float dn = __shfl_down_sync(FULL, tot, 1 << l);
        if (lane + (1 << l) < 32) tot = fmaf(Bl[l], dn, tot);
    }
    float P = __shfl_down_sync(FULL, tot, 1);
    if (lane == 31) P = 0.0f;
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = fmaf(dk[E - 1 - k], P, v[k]);
}

struct Tables {
    float Bl[5], dk[E], Bw[E];  // dec^(8*2^l), dec^(k+1), dec^(8L+k+1)
};

__device__ __forceinline__ Tables make_tables(double dec, int lane) {
    Tables tb;
    const df d{(float)dec, (float)(dec - (double)(float)dec)};
    df u = d, b = df_pow(d, 8 * lane + 1);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        tb.dk[k] = u.hi;
        tb.Bw[k] = b.hi;
        u = df_mul(u, d);
        b = df_mul(b, d);
    }
    df d8 = df_pow(d, 8);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        tb.Bl[l] = d8.hi;
        d8 = df_mul(d8, d8);
    }
    return tb;
}

__device__ __forceinline__ void load_diff(float (&dv)[E], const uint32_t *xb, const uint32_t *yb, long long w,
                                          int cnt, int lane) {
    const int t0 = 8 * lane;
    const long long widx = (w >> 5) + (t0 >> 5);
    const uint32_t xw = (t0 < cnt) ? (xb[widx] >> (t0 & 31)) & 0xffu : 0u;
    const uint32_t yw = (t0 < cnt) ? (yb[widx] >> (t0 & 31)) & 0xffu : 0u;
#pragma unroll
    for (int k = 0; k < E; ++k)
        dv[k] = (t0 + k < cnt) ? (float)((xw >> k) & 1u) - (float)((yw >> k) & 1u) : 0.0f;
}

// Forward filter: loss[r] (double-single summed) and f entering each chunk.
__global__ void __launch_bounds__(WARPS * 32) vr_forward_kernel(long long rows, long long T, const uint32_t *x,
                                                                 const uint32_t *y, double dec, double scale,
                                                                 long long chunk, long long nchunk, float *f_ckpt,
                                                                 float *loss) {
    const int lane = threadIdx.x & 31;
    const long long r = (long long)blockIdx.x * WARPS + (threadIdx.x >> 5);
    if (r >= rows) return;
    const Tables tb = make_tables(dec, lane);
    const long long nw = (T + 31) / 32;
    const uint32_t *xb = x + r * nw, *yb = y + r * nw;
    float fin = 0.0f;
    df acc{0.0f, 0.0f};
    for (long long w = 0; w < T; w += WIN) {
        if (f_ckpt && w % chunk == 0 && lane == 0) f_ckpt[r * nchunk + w / chunk] = fin;
        const int cnt = (int)(T - w < WIN ? T - w : WIN);
        float f[E];
        load_diff(f, xb, yb, w, cnt, lane);
        scan_fwd(f, tb.dk[0], tb.Bl, tb.dk, lane);
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            f[k] = fmaf(tb.Bw[k], fin, f[k]);
            if (8 * lane + k < cnt) s = fmaf(f[k], f[k], s);
        }
        acc = df_add(acc, df{s, 0.0f});
        const int tl = cnt - 1, kl = tl & 7;
        float mine = f[0];
#pragma unroll
        for (int k = 1; k < E; ++k)
            if (k == kl) mine = f[k];
        fin = __shfl_sync(FULL, mine, tl >> 3);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const df o{__shfl_xor_sync(FULL, acc.hi, off), __shfl_xor_sync(FULL, acc.lo, off)};
        acc = df_add(acc, o);
    }
    if (lane == 0 && loss) loss[r] = (float)(scale * ((double)acc.hi + (double)acc.lo));
}

// Gradient for steps [t0, t1) (t0 a multiple of 256 and of the chunk start):
// grad[r, t - t0] = (2 DT / tau_R) g[t], g carried from t1 in g_carry (updated).
__global__ void __launch_bounds__(WARPS * 32) vr_backward_kernel(long long rows, long long T, const uint32_t *x,
                                                                  const uint32_t *y, double dec, float gscale,
                                                                  long long t0, long long t1, const float *f_start,
                                                                  float *g_carry, float *grad, long long ldg) {
    extern __shared__ float fsm[];  // f entering each window of the chunk, per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long r = (long long)blockIdx.x * WARPS + warp;
    if (r >= rows) return;
    const Tables tb = make_tables(dec, lane);
    const long long nw = (T + 31) / 32;
    const uint32_t *xb = x + r * nw, *yb = y + r * nw;
    const int nwin = (int)((t1 - t0 + WIN - 1) / WIN);
    float *fw = fsm + warp * nwin;
    float fin = f_start[r];
    for (int wi = 0; wi < nwin; ++wi) {  // f entering each window
        const long long w = t0 + (long long)wi * WIN;
        if (lane == 0) fw[wi] = fin;
        const int cnt = (int)(t1 - w < WIN ? t1 - w : WIN);
        float f[E];
        load_diff(f, xb, yb, w, cnt, lane);
        scan_fwd(f, tb.dk[0], tb.Bl, tb.dk, lane);
#pragma unroll
        for (int k = 0; k < E; ++k) f[k] = fmaf(tb.Bw[k], fin, f[k]);
        const int tl = cnt - 1, kl = tl & 7;
        float mine = f[0];
#pragma unroll
        for (int k = 1; k < E; ++k)
            if (k == kl) mine = f[k];
        fin = __shfl_sync(FULL, mine, tl >> 3);
    }
    __syncwarp();
    float gc = g_carry[r];
    for (int wi = nwin - 1; wi >= 0; --wi) {
        const long long w = t0 + (long long)wi * WIN;
        const int cnt = (int)(t1 - w < WIN ? t1 - w : WIN);
        float f[E];
        load_diff(f, xb, yb, w, cnt, lane);
        scan_fwd(f, tb.dk[0], tb.Bl, tb.dk, lane);
        const float fs = fw[wi];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            f[k] = fmaf(tb.Bw[k], fs, f[k]);
            if (8 * lane + k >= cnt) f[k] = 0.0f;
            if (8 * lane + k == cnt - 1) f[k] = fmaf(tb.dk[0], gc, f[k]);  // carry from step w + cnt
        }
        scan_rev(f, tb.dk[0], tb.Bl, tb.dk, lane);
        float *go = grad + r * ldg + (w - t0) + 8 * lane;
#pragma unroll
        for (int k = 0; k < E; ++k)
            if (8 * lane + k < cnt) go[k] = gscale * f[k];
        gc = __shfl_sync(FULL, f[0], 0);
    }
    if (lane == 0) g_carry[r] = gc;
}

}  // namespace vr

int launch_vr_forward(long long rows, long long T, const uint32_t *x, const uint32_t *y, double dec, double scale,
                      long long chunk, float *f_ckpt, float *loss, cudaStream_t st) {
    const long long nchunk = (T + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((rows + vr::WARPS - 1) / vr::WARPS);
    if (grid == 0) return 0;
    vr::vr_forward_kernel<<<grid, vr::WARPS * 32, 0, st>>>(rows, T, x, y, dec, scale, chunk, nchunk, f_ckpt, loss);
    return (int)cudaGetLastError();
}

int launch_vr_backward(long long rows, long long T, const uint32_t *x, const uint32_t *y, double dec, float gscale,
                       long long t0, long long t1, const float *f_start, float *g_carry, float *grad, long long ldg,
                       cudaStream_t st) {
    const unsigned grid = (unsigned)((rows + vr::WARPS - 1) / vr::WARPS);
    if (grid == 0) return 0;
    const int nwin = (int)((t1 - t0 + vr::WIN - 1) / vr::WIN);
    const size_t smem = (size_t)vr::WARPS * nwin * sizeof(float);
    vr::vr_backward_kernel<<<grid, vr::WARPS * 32, smem, st>>>(rows, T, x, y, dec, gscale, t0, t1, f_start, g_carry,
                                                               grad, ldg);
    return (int)cudaGetLastError();
}

}  // namespace alif
