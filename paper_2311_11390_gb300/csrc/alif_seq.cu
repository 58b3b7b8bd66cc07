// Plain sequential ALIF kernels: the standard model (Section 2, Eqs 1-5) as a
// GPU kernel that walks time one step at a time, one thread per neuron row.
// They are the comparator of the blocked kernels ("standard SNN", Section 4.1):
// no shared-memory staging, no manual unrolling, FP32 state.
#include "common.cuh"

namespace alif {
namespace seq {

struct FwdArgs {
    long long rows, N, T, nwords;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    uint32_t *spikes;
    float *vtr, *atr;
    AlifState *fin;
};

__global__ void fwd_seq_kernel(const FwdArgs A) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.rows) return;
    const AlifNeuron nr = A.nrn[r % A.N];
    AlifState s{0.0f, 0.0f, 0};
    if (A.init) s = A.init[r];
    int rem = s.rem > 0 ? s.rem : 0;
    float v = rem > 0 ? 0.0f : s.v;  // V[t-1] after the reset of Eq 2
    float a = s.a;                   // a[t]
    uint32_t word = 0;
    const float *I = A.I + r * A.T;
    for (long long t = 0; t < A.T; ++t) {
        const float Iin = rem == 0 ? I[t] : 0.0f;          // Eq 4
        const float V = nr.beta_hi * v + nr.c_hi * Iin;    // Eq 2
        const float theta = nr.theta0 + nr.d * a;          // Eq 5
        const bool S = V > theta;                          // Eq 1
        if (A.vtr) A.vtr[r * A.T + t] = V;
        if (A.atr) A.atr[r * A.T + t] = a;
        if (S) {
            v = 0.0f;
            rem = nr.teff - 1;
        } else {
            v = V;
            rem = rem > 0 ? rem - 1 : 0;
        }
        a = nr.p_hi * a + (S ? 1.0f : 0.0f);
        word |= (S ? 1u : 0u) << (t & 31);
        if ((t & 31) == 31 || t == A.T - 1) {
            A.spikes[r * A.nwords + (t >> 5)] = word;
            word = 0;
        }
    }
    if (A.fin) {
        AlifState f;
        f.v = v;
        f.a = a;
        f.rem = rem;
        A.fin[r] = f;
    }
}

// Tuned sequential forward: the same per-step recurrence as fwd_seq_kernel,
// with the input staged so that global loads are coalesced.  A warp owns 32
// consecutive rows (lane = row); every 32 steps it reads the [32 rows x 32
// steps] tile as 32 coalesced 128-byte row segments (lane = step), passes it
// through a padded shared tile, and issues the next tile's loads before it
// walks the current one.
constexpr int SEQ_WARPS = 4;
__global__ void __launch_bounds__(SEQ_WARPS * 32) fwd_seq_staged_kernel(const FwdArgs A) {
    __shared__ float tile[SEQ_WARPS][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = ((long long)blockIdx.x * SEQ_WARPS + warp) * 32;
    if (r0 >= A.rows) return;
    const long long r = r0 + lane;
    const bool live = r < A.rows;
    const int nrows = (int)(A.rows - r0 < 32 ? A.rows - r0 : 32);
    const AlifNeuron nr = A.nrn[(live ? r : r0) % A.N];
    AlifState s{0.0f, 0.0f, 0};
    if (A.init && live) s = A.init[r];
    int rem = s.rem > 0 ? s.rem : 0;
    float v = rem > 0 ? 0.0f : s.v;
    float a = s.a;
    float nxt[32];
    auto load = [&](long long tb) {
        const bool in = tb + lane < A.T;
#pragma unroll
        for (int j = 0; j < 32; ++j) nxt[j] = (j < nrows && in) ? __ldg(A.I + (r0 + j) * A.T + tb + lane) : 0.0f;
    };
    load(0);
    for (long long tb = 0; tb < A.T; tb += 32) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[warp][j][lane] = nxt[j];
        __syncwarp();
        if (tb + 32 < A.T) load(tb + 32);
        const int n = (int)(A.T - tb < 32 ? A.T - tb : 32);
        uint32_t word = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k < n) {
                const float Iin = rem == 0 ? tile[warp][lane][k] : 0.0f;  // Eq 4
                const float V = nr.beta_hi * v + nr.c_hi * Iin;           // Eq 2
                const float theta = nr.theta0 + nr.d * a;                 // Eq 5
                const bool S = V > theta;                                 // Eq 1
                if (live && A.vtr) A.vtr[r * A.T + tb + k] = V;
                if (live && A.atr) A.atr[r * A.T + tb + k] = a;
                if (S) {
                    v = 0.0f;
                    rem = nr.teff - 1;
                } else {
                    v = V;
                    rem = rem > 0 ? rem - 1 : 0;
                }
                a = nr.p_hi * a + (S ? 1.0f : 0.0f);
                word |= (S ? 1u : 0u) << k;
            }
        }
        if (live) A.spikes[r * A.nwords + (tb >> 5)] = word;
    }
    if (A.fin && live) {
        AlifState f;
        f.v = v;
        f.a = a;
        f.rem = rem;
        A.fin[r] = f;
    }
}

struct BwdArgs {
    long long rows, N, T, nwords;
    const float *I;
    const AlifNeuron *nrn;
    const AlifState *init;
    const uint32_t *spikes;
    const float *vtr, *atr;
    const float *gS, *gV, *ga, *gfin;
    float slope;
    float *gI, *ginit;
    float *part;  // [rows, 5] per-row parameter gradients
};

__device__ __forceinline__ int spike_at(const uint32_t *bits, long long t) {
    return (bits[t >> 5] >> (t & 31)) & 1u;
}

// Largest tau <= from with a spike, or -1.
__device__ long long prev_spike(const uint32_t *bits, long long from) {
    while (from >= 0) {
        const uint32_t wd = bits[from >> 5] & (0xffffffffu >> (31 - (from & 31)));
        if (wd) return (from & ~31LL) + 31 - __clz(wd);
        from = (from & ~31LL) - 1;
    }
    return -1;
}

__global__ void bwd_seq_kernel(const BwdArgs A) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.rows) return;
    const AlifNeuron nr = A.nrn[r % A.N];
    AlifState s{0.0f, 0.0f, 0};
    if (A.init) s = A.init[r];
    const int rem0 = s.rem > 0 ? s.rem : 0;
    const float v0 = rem0 > 0 ? 0.0f : s.v;
    const uint32_t *bits = A.spikes + r * A.nwords;
    const long long base = r * A.T;
    const float beta = nr.beta_hi, p = nr.p_hi, c = nr.c_hi, d = nr.d;

    float gVn = A.gfin ? A.gfin[2 * r] : 0.0f;      // dL/d(final v)
    float gan = A.gfin ? A.gfin[2 * r + 1] : 0.0f;  // dL/da[t+1]
    float g_th0 = 0.0f, g_d = 0.0f, g_beta = 0.0f, g_p = 0.0f, g_R = 0.0f;
    long long last = prev_spike(bits, A.T - 2);      // last spike before t = T-1
    for (long long t = A.T - 1; t >= 0; --t) {
        if (last == t) last = prev_spike(bits, t - 1);  // keep "last spike < t"
        const int S = spike_at(bits, t);
        const float V = A.vtr[base + t], a = A.atr[base + t];
        const int adm = (last >= 0) ? (t - last >= nr.teff) : (t >= rem0);
        const float Iin = adm ? A.I[base + t] : 0.0f;
        const float vprev = (t == 0) ? v0 : ((last == t - 1) ? 0.0f : A.vtr[base + t - 1]);
        const float u = V - (nr.theta0 + d * a);
        const float den = A.slope * fabsf(u) + 1.0f;
        const float sg = 1.0f / (den * den);
        const float gs = A.gS[base + t];
        // dL/dV[t]: spike and trace terms plus the path into step t+1 (reset detached)
        const float next = (t == A.T - 1) ? (S ? 0.0f : gVn) : (S ? 0.0f : beta * gVn);
        const float GV = sg * gs + (A.gV ? A.gV[base + t] : 0.0f) + next;
        const float Gth = -sg * gs;
        const float Ga = d * Gth + (A.ga ? A.ga[base + t] : 0.0f) + p * gan;
        if (A.gI) A.gI[base + t] = c * (adm ? 1.0f : 0.0f) * GV;
        g_th0 += Gth;
        g_d += a * Gth;
        g_beta += (vprev - nr.R * Iin) * GV;
        g_p += a * gan;  // a[t+1] = p a[t] + S[t]
        g_R += nr.one_minus_beta * Iin * GV;
        gVn = GV;
        gan = Ga;
    }
    if (A.ginit) {
        A.ginit[2 * r] = beta * gVn;
        A.ginit[2 * r + 1] = gan;
    }
    float *o = A.part + r * (2 * ALIF_NUM_PARAM_GRADS);  // (value, 0) pairs
    o[2 * ALIF_G_TAU_MEM] = g_beta * nr.dbeta_dtau;
    o[2 * ALIF_G_TAU_ADAPT] = g_p * nr.dp_dtau;
    o[2 * ALIF_G_THETA0] = g_th0;
    o[2 * ALIF_G_D] = g_d;
    o[2 * ALIF_G_R] = g_R;
#pragma unroll
    for (int k = 0; k < ALIF_NUM_PARAM_GRADS; ++k) o[2 * k + 1] = 0.0f;
}

}  // namespace seq

int launch_alif_forward_seq(long long B, long long N, long long T, const float *I,
                            const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                            float *vtr, float *atr, AlifState *fin, cudaStream_t stream) {
    seq::FwdArgs A{B * N, N, T, (T + 31) / 32, I, nrn, init, spikes, vtr, atr, fin};
    const int threads = 128;
    const long long blocks = (A.rows + threads - 1) / threads;
    if (blocks <= 0) return 0;
    seq::fwd_seq_kernel<<<(unsigned)blocks, threads, 0, stream>>>(A);
    return (int)cudaGetLastError();
}

int launch_alif_forward_seq_staged(long long B, long long N, long long T, const float *I,
                                   const AlifNeuron *nrn, const AlifState *init, uint32_t *spikes,
                                   float *vtr, float *atr, AlifState *fin, cudaStream_t stream) {
    seq::FwdArgs A{B * N, N, T, (T + 31) / 32, I, nrn, init, spikes, vtr, atr, fin};
    const long long per_block = 32LL * seq::SEQ_WARPS;
    const long long blocks = (A.rows + per_block - 1) / per_block;
    if (blocks <= 0) return 0;
    seq::fwd_seq_staged_kernel<<<(unsigned)blocks, seq::SEQ_WARPS * 32, 0, stream>>>(A);
    return (int)cudaGetLastError();
}

int launch_alif_backward_seq(long long B, long long N, long long T, const float *I,
                             const AlifNeuron *nrn, const AlifState *init, const uint32_t *spikes,
                             const float *vtr, const float *atr, const float *gS, const float *gV,
                             const float *ga, const float *gfin, float slope, float *gI,
                             float *ginit, float *part, cudaStream_t stream) {
    seq::BwdArgs A{B * N, N, T, (T + 31) / 32, I, nrn, init, spikes, vtr, atr,
                   gS, gV, ga, gfin, slope, gI, ginit, part};
    const int threads = 128;
    const long long blocks = (A.rows + threads - 1) / threads;
    if (blocks <= 0) return 0;
    seq::bwd_seq_kernel<<<(unsigned)blocks, threads, 0, stream>>>(A);
    return (int)cudaGetLastError();
}

}  // namespace alif
