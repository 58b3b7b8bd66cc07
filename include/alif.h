/*
 * alif.h -- C ABI of the GB300 (sm_103a) ARP-blocked ALIF library.
 *
 * Implements the hot path of Taylor, King & Harper, "Addressing the
 * speed-accuracy simulation trade-off for adaptive spiking neurons"
 * (NeurIPS 2023): simulation of adaptive leaky integrate-and-fire (ALIF)
 * neurons (Section 2, Eqs 1-5) with the absolute-refractory-period blocked
 * reformulation (Section 3, Props 1-5), its surrogate-gradient backward
 * (Supplementary, "Surrogate gradient", "Detaching gradients"), and the
 * feedforward synaptic projection that produces the input current (Eq 3,
 * Prop 3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every entry point returns an int status: ALIF_OK (0) or a negative code.
 *    alif_last_error() gives a message for the calling thread.  No exception
 *    crosses the ABI and nothing calls exit().
 *  - Pointers are DEVICE pointers owned by the caller unless a comment says
 *    "host".  The library allocates no device memory on any compute call;
 *    scratch space comes from a caller buffer sized by a *_workspace_size()
 *    query.  It calls no other library's kernels.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream and never synchronise the host.
 *  - Arrays are dense row-major in the shapes given.  "Row" means one
 *    (batch b, neuron i) pair, row index b*N + i; time is the fastest axis.
 *  - Time steps are indexed t = 0..T-1 for the paper's t = 1..T.
 *  - Spike trains are bit-packed: uint32 [rows, ceil(T/32)], bit t%32 of word
 *    t/32, least significant bit first.  Bits at t >= T are written as zero.
 *  - A device-side wait that exceeds its time limit (about one second) does
 *    not hang: the kernel records ALIF_ETIMEOUT in a device status word and
 *    returns; read and clear it with alif_device_status().
 *
 * Model (Eqs 1-5, state form).  Per row, with beta = exp(-DT/tau_mem),
 * p = exp(-DT/tau_adapt), T_R = ARP/DT and T_eff = max(T_R, 2):
 *     V[t]  = beta * v + (1 - beta) * R * I[t] * m[t]      (Eq 2, Eq 4)
 *     theta = theta0 + d * a[t]                           (Eq 5)
 *     S[t]  = V[t] > theta                                (Eq 1, strict)
 * where v is V[t-1] with the reset of Eq 2 applied (0 after a spike) and
 * m[t] = 1 once T_eff steps have passed since the last spike (the ARP of
 * Eq 4; T_R = 1 behaves as 2 because the reset already zeroes the step after
 * a spike).  Then a[t+1] = p a[t] + S[t].
 */
#ifndef ALIF_H
#define ALIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define ALIF_OK            0
#define ALIF_EINVAL       -1   /* null pointer, non-finite or out-of-range parameter */
#define ALIF_ETR          -2   /* ARP/DT is not an integer >= 1 (to 1e-9 relative)   */
#define ALIF_ESHAPE       -3   /* negative or overflowing size, misaligned pointer    */
#define ALIF_EUNSUPPORTED -4   /* valid request the library does not serve            */
#define ALIF_ECUDA        -5   /* a CUDA runtime call failed                          */
#define ALIF_ETIMEOUT     -6   /* a device-side bounded wait expired                  */
#define ALIF_EWORKSPACE   -7   /* workspace pointer/size too small                    */

/* Time steps between saved states: the forward saves the state entering
 * steps 0, 256, 512, ... (the block-boundary checkpoint the backward reads). */
#define ALIF_CKPT_STEPS 256

/* Neuron state entering step t (12 bytes):
 *   v   = V[t-1] * (1 - S[t-1])  (the reset of Eq 2 applied; must be 0 if rem > 0)
 *   a   = a[t]                   (adaptation of Eq 5 at step t, spike of t-1 included)
 *   rem = steps still masked by the ARP: input is admitted from step t + rem on.
 * The rest state is {0, 0, 0}. */
typedef struct AlifState {
    float v;
    float a;
    int32_t rem;
} AlifState;

/* Per-neuron constants prepared on the host in FP64 by alif_prepare() and
 * rounded once to FP32 (64 bytes).  x_hi + x_lo is an unevaluated sum that
 * carries the FP64 value to ~2^-48 relative; kernels use x_hi on the fast
 * path and the pair where exact decisions are needed. */
typedef struct AlifNeuron {
    float beta_hi, beta_lo;   /* beta = exp(-DT / tau_mem)          (Eq 2)   */
    float p_hi, p_lo;         /* p = exp(-DT / tau_adapt)           (Eq 5)   */
    float c_hi, c_lo;         /* (1 - beta) * R, the input gain of Eq 2      */
    float theta0, d;          /* threshold baseline and adaptation scale     */
    float R;                  /* input resistance (1 = paper's normalisation) */
    float one_minus_beta;     /* 1 - beta                                    */
    float dbeta_dtau;         /* beta * DT / tau_mem^2                       */
    float dp_dtau;            /* p * DT / tau_adapt^2                        */
    float guard;              /* reserved, written as 0                      */
    int32_t tr;               /* T_R                                         */
    int32_t teff;             /* max(T_R, 2)                                 */
    int32_t reserved;
} AlifNeuron;

/* Order of the per-neuron parameter gradients written by alif_backward(). */
enum { ALIF_G_TAU_MEM = 0, ALIF_G_TAU_ADAPT = 1, ALIF_G_THETA0 = 2, ALIF_G_D = 3,
       ALIF_G_R = 4, ALIF_NUM_PARAM_GRADS = 5 };

/* ------------------------------------------------------------- utilities */

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to len) into buf (host).  Returns the full message length. */
int alif_last_error(char *buf, size_t len);

/* Reads the device status word (ALIF_OK, ALIF_ETIMEOUT, or ALIF_EUNSUPPORTED
 * for an event-bucket overflow of alif_forward_fused) into *status_host and
 * clears it.  Synchronises `stream`. */
int alif_device_status(void *stream, int32_t *status_host);

/* T_R = ARP/DT rounded to the nearest integer (Section 3.2 blocks span the
 * ARP).  Returns T_R >= 1, or ALIF_ETR when |ARP/DT - T_R| > 1e-9 max(1, ARP/DT)
 * or T_R < 1, or ALIF_EINVAL for non-positive / non-finite arguments. */
int alif_tr(double dt_ms, double arp_ms);

/* Host preparation (all pointers HOST).  For each neuron i computes, in FP64,
 * beta = exp(-DT/tau_mem[i]) and p = exp(-DT/tau_adapt[i]) (Supplementary,
 * "Weight initialisation"; no clamping is applied), the gain (1-beta) R[i],
 * and the derivative factors used to chain gradients to the time constants;
 * writes out[N].  R may be NULL (all 1).
 * Rejects (ALIF_EINVAL) tau <= 0, theta0 <= 0, d < 0, R < 0 or non-finite
 * values: theta0 > 0 and d >= 0 keep theta > 0 = V during the ARP, which the
 * blocked reformulation (Prop 3) relies on.  Returns ALIF_OK or an error. */
int alif_prepare(int64_t N, const float *tau_mem, const float *tau_adapt,
                 const float *theta0, const float *d_adapt, const float *R,
                 double dt_ms, double arp_ms, AlifNeuron *out);

/* Number of saved states per row: ceil(T / ALIF_CKPT_STEPS) (0 for T = 0). */
int64_t alif_ckpt_count(int64_t T);

/* ------------------------------------------------------- block forward  */

/* alif_prepare() (host, once per parameter set) followed by alif_forward()
 * together form the forward of the problem statement (currents, per-neuron
 * tau_mem / tau_adapt / theta0 / d / R, DT, ARP -> spikes and traces). */

/* ARP-blocked forward (Section 3, Props 1-5; Eqs 1-5).
 *   I        [B,N,T] float   input current (already including bias, Eq 3)
 *   neurons  [N] AlifNeuron  from alif_prepare(), copied to the device
 *   init     [B,N] AlifState initial state, or NULL for rest
 *   spikes   [B,N,ceil(T/32)] uint32 output spike bits (required)
 *   v_trace  [B,N,T] float   membrane potential V[t] (Eq 2), or NULL
 *   a_trace  [B,N,T] float   adaptation a[t] (Eq 5), or NULL
 *   ckpt     [B,N,alif_ckpt_count(T)] AlifState: state entering step 256k, or NULL
 *            (alif_backward needs it)
 *   final_state [B,N] AlifState state entering step T, or NULL
 * With B*N >= 32 x the SM count (and no traces), a lane takes a row and walks
 * it through Blocks of K <= T_eff steps (K = 16, 8, 4 or 2): the Block's
 * no-reset membrane (Prop 1) from an input-only chain, its first crossing
 * (Prop 2, Eq 9), and the state carried to the next Block (Props 3-5).  With
 * fewer rows, or with traces, a warp takes a row: inside each 256- or 512-step
 * window the no-reset membrane is a parallel decayed scan, the first crossing
 * is found with a warp ballot, and after a spike the next search starts T_eff
 * steps later (the ARP mask of Prop 3) with the membrane reset (Prop 4) and
 * the adaptation carried in closed form (Prop 5).  alif_forward_layout() and
 * alif_forward_window() force either choice.  In both, spike decisions whose
 * FP32 margin lies within an error bound counted from the kernel's own
 * roundings are re-decided in double-single arithmetic from an exact anchor,
 * so the spikes equal the FP64 standard model's except at ties far below FP32
 * resolution.  I must be 4-byte aligned; 16-byte alignment with T % 4 == 0
 * enables the bulk-copy path (and is required for the lane layout). */
int alif_forward(int64_t B, int64_t N, int64_t T, const float *I,
                 const AlifNeuron *neurons, const AlifState *init,
                 uint32_t *spikes, float *v_trace, float *a_trace,
                 AlifState *ckpt, AlifState *final_state, void *stream);

/* Workspace bytes alif_forward_fused() needs: per-step event offsets and the
 * event buckets of every (batch element, 32-step word), max_events_per_word
 * entries each. */
size_t alif_forward_fused_workspace_size(int64_t B, int64_t Nin, int64_t T, int32_t max_events_per_word);

/* Synaptic projection fused into the block forward (the feedforward term of
 * Eq 3 / Prop 3 feeding Section 3's Blocks): the currents
 *     I[b, i, t] = bias[i] + sum over the inputs j active at (b, t) of W[i, j]
 * are computed inside the forward from the input events, with the exact FP32
 * weights summed in ascending input order (within (k+1) 2^-24 (|bias_i| +
 * sum_j |W_ij| S_j) of the exact sum for k active inputs), written to I (the
 * backward's input), and simulated as alif_forward() does.  A first kernel
 * turns the raster into event buckets: per (batch element, 32-step word) the
 * per-step offsets and the active inputs, at most max_events_per_word of them
 * (a word with more records ALIF_EUNSUPPORTED in the device status word, and
 * its currents are then incomplete).
 *   W      [N, Nin] FP32 weights (Nin <= 1024, else ALIF_EUNSUPPORTED)
 *   S_in   [B, Nin, ceil(T/32)] input spike bits; bias [N] or NULL
 *   I      [B, N, T] output currents (16-byte aligned)
 *   neurons, init, spikes, ckpt, final_state: as alif_forward()
 *   workspace (256-byte aligned) >= alif_forward_fused_workspace_size(...). */
int alif_forward_fused(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W, const uint32_t *S_in,
                       const float *bias, const AlifNeuron *neurons, const AlifState *init,
                       int32_t max_events_per_word, float *I, uint32_t *spikes, AlifState *ckpt,
                       AlifState *final_state, void *workspace, size_t workspace_bytes, void *stream);

/* Window length of alif_forward (host; a performance choice: spikes, traces
 * and checkpoints are the same).  0, the default: 512-step windows (three CTAs
 * of four warps per SM) when B * N <= 8 x the SM count, where warp slots stay
 * empty and each row's chain of windows sets the time, and 256-step windows
 * (four CTAs per SM) otherwise.  256 or 512 forces one.  The 512-step kernel
 * serves calls on the TMA path (T a multiple of 16, 16-byte aligned) without
 * traces; other calls use 256.  Process-wide, not synchronised.  Returns the
 * previous setting, or ALIF_EINVAL (setting unchanged) for any other value. */
int alif_forward_window(int steps);

/* Layout of alif_forward (host; a performance choice: the spikes are the same,
 * checkpoints and final states agree within FP32 rounding).  0, the default: a
 * lane per row when B * N >= 32 x the SM count, a warp per row otherwise.
 * 1: a warp per row (the windows above).  2: a lane per row: each lane walks its
 * row through Blocks of K <= T_R steps (K = 8, 4 or 2 by the smallest T_eff of
 * the warp's 32 rows), at most one spike per Block (Section 3.1), with the
 * Block's no-reset membrane, thresholds and first crossing computed as
 * independent operations inside the lane (Props 1-5) and the membrane carried
 * in double-single between Blocks; input staged by TMA as [32 rows x 64 steps]
 * tiles.  The lane layout serves calls without traces with T % 4 == 0 and I
 * 16-byte aligned; other calls use a warp per row.  Process-wide, not
 * synchronised.  Returns the previous setting, or ALIF_EINVAL (setting
 * unchanged) for any other value. */
int alif_forward_layout(int layout);

/* Counters of the last alif_forward on this device (host out[4]): fast-path
 * decisions re-checked exactly, of which spikes, and rows processed.  Reads
 * and clears device counters; synchronises `stream`. */
int alif_forward_stats(void *stream, int64_t *out4);

/* ------------------------------------------------------- block backward */

/* Workspace bytes alif_backward() needs: per-row partial parameter sums as
 * double-single (hi, lo) float pairs, B * N * 10 * 4 bytes. */
size_t alif_backward_workspace_size(int64_t B, int64_t N);

/* Surrogate-gradient backward of alif_forward, gradients "detached" as in the
 * Supplementary ("Detaching gradients"): S[t-1] is a constant in the reset of
 * Eq 2 and in the update of Eq 5, the ARP mask has no gradient, and dS/dV is
 * the fast sigmoid 1/(slope |V - theta| + 1)^2 evaluated at u = V - theta,
 * reaching theta as -dS/du.  Walks windows of 256 (or 512, see
 * alif_backward_window) steps in reverse, recomputing V and a inside each
 * window from `ckpt` and the stored spikes.
 *   I, neurons, init, spikes, ckpt   as given to / produced by alif_forward
 *   grad_spikes [B,N,T] float  dL/dS (required)
 *   grad_v, grad_a [B,N,T]     dL/dV, dL/da of the traces, or NULL
 *   grad_final  [B,N,2] float  dL/d(final v, final a), or NULL
 *   grad_I      [B,N,T] float  output dL/dI, or NULL (parameter fits)
 *   grad_init   [B,N,2] float  output dL/d(init v, init a), or NULL
 *   grad_params [5,N] float    output, summed over the batch in a fixed order
 *                              (deterministic): tau_mem, tau_adapt, theta0, d, R
 *   workspace, workspace_bytes  >= alif_backward_workspace_size(B, N)
 */
int alif_backward(int64_t B, int64_t N, int64_t T, const float *I,
                  const AlifNeuron *neurons, const AlifState *init,
                  const uint32_t *spikes, const AlifState *ckpt,
                  const float *grad_spikes, const float *grad_v, const float *grad_a,
                  const float *grad_final, float slope,
                  float *grad_I, float *grad_init, float *grad_params,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Window length of alif_backward and alif_backward_surrogate (host; a
 * performance choice, the results agree within rounding).  0, the default:
 * 512-step windows (two CTAs of four warps per SM) when B * N <= 8 x the SM
 * count, where warp slots stay empty and each row's chain of windows sets the
 * time, and 256-step windows (four CTAs per SM) otherwise.  256 or 512 forces
 * one.  The 512-step kernel serves calls whose tensors take the TMA path (T a
 * multiple of 16, 16-byte aligned) without grad_v / grad_a; other calls use
 * 256.  Process-wide, not synchronised: set it before launching from several
 * threads.  Returns the previous setting, or ALIF_EINVAL (setting unchanged)
 * for any other value. */
int alif_backward_window(int steps);

/* The surrogates of the Supplementary's comparison ("Surrogate gradient"),
 * evaluated at u = V - theta:
 *   ALIF_SG_FAST_SIGMOID   1/(k|u|+1)^2 with slope k (the `slope` argument)
 *   ALIF_SG_MULTI_GAUSSIAN 1.15 N(u|0, 0.5^2) - 0.15 N(u|3, 3^2) - 0.15 N(u|-3, 3^2)
 *                          (N the normal density; means and variances as printed)
 *   ALIF_SG_BOXCAR         0.5 where |u| <= 0.5, else 0                              */
enum { ALIF_SG_FAST_SIGMOID = 0, ALIF_SG_MULTI_GAUSSIAN = 1, ALIF_SG_BOXCAR = 2 };

/* alif_backward with a choice of surrogate (`slope` is used by the fast sigmoid
 * only); ALIF_EINVAL for an unknown surrogate.  Otherwise identical. */
int alif_backward_surrogate(int64_t B, int64_t N, int64_t T, const float *I,
                            const AlifNeuron *neurons, const AlifState *init,
                            const uint32_t *spikes, const AlifState *ckpt,
                            const float *grad_spikes, const float *grad_v, const float *grad_a,
                            const float *grad_final, int surrogate, float slope,
                            float *grad_I, float *grad_init, float *grad_params,
                            void *workspace, size_t workspace_bytes, void *stream);

/* alif_backward_surrogate with "attached" gradients (Supplementary, "Detaching
 * gradients"): the spike S[t] also carries its surrogate gradient where it enters
 * the next step, through the reset factor of V[t+1] (Eq 2) and the update
 * a[t+1] = p a[t] + S[t] (Eq 5); the ARP mask of Eq 4 still carries none.  The
 * reverse recurrences of G_V and G_a are then coupled through
 *   dL/dS[t] = gS[t] + G_a[t+1] - (beta V[t] + (1 - beta) R m[t+1] I[t+1]) G_V[t+1].
 * Arguments, layouts, outputs and errors as alif_backward_surrogate(), plus:
 *   grad_final_spike  [B, N] device, nullable (= 0): added to dL/dS of the last
 *                     step; pass the grad_init_spike of the call that continues
 *                     this sequence (the state (v, a) carries V after its reset,
 *                     so the input term of the bracket above crosses the call
 *                     boundary here);
 *   grad_init_spike   [B, N] device, nullable: -(1 - beta) R m[0] I[0] G_V[0],
 *                     the part of dL/dS of the step before this call that comes
 *                     through this call's first input.
 * grad_final couples to the last step through the final state (v, a) =
 * (V (1 - S), p a + S). */
int alif_backward_attached(int64_t B, int64_t N, int64_t T, const float *I,
                           const AlifNeuron *neurons, const AlifState *init,
                           const uint32_t *spikes, const AlifState *ckpt,
                           const float *grad_spikes, const float *grad_v, const float *grad_a,
                           const float *grad_final, const float *grad_final_spike,
                           int surrogate, float slope,
                           float *grad_I, float *grad_init, float *grad_init_spike,
                           float *grad_params, void *workspace, size_t workspace_bytes,
                           void *stream);

/* ------------------------------------------------- recurrent layer    */

/* Recurrent ALIF layer with transmission latency D = T_R (Section 2: the
 * input current of Eq 3 has a recurrent term sum_j W_rec[i][j] S_j[t - D], and
 * D is taken equal to the ARP; Prop 3 gives Block n+1 its recurrent current
 * from the spikes of Block n):
 *     I[b,i,t] = I_ff[b,i,t] + sum_j W_rec[i][j] S[b,j,t - T_R]   (0 for t < T_R),
 * then the model above.  A batch element's neurons exchange spikes once per T_R
 * steps.  No spike before step 0 is assumed (init sets only each neuron's own
 * state).
 *   I_ff        [B, N, T] device: bias + feedforward current (syn_project output).
 *   W_rec_t     [N, N] device: W_rec TRANSPOSED, row j = the weights of
 *               presynaptic neuron j onto every i (syn_transpose_weights of W_rec).
 *   neurons     table from alif_prepare with the same dt_ms / arp_ms.
 *   dt_ms, arp_ms  give T_R = ARP/DT (as alif_tr; ALIF_ETR otherwise).
 *   I_total     [B, N, T] device, nullable: I_ff + recurrent current, the input
 *               the backward needs; may be I_ff itself (updated in place).
 *   spikes, ckpt, final_state, init: as alif_forward().
 * Spike decisions are exact for the FP32 total current (double-single state),
 * so alif_forward() on I_total returns the same spikes.  Needs N <= 8192 and
 * T_R <= 1023 within ~200 KB of shared memory per 1024 neurons (ALIF_EUNSUPPORTED
 * otherwise).  Gradients ("detached": the recurrent synapses carry no gradient
 * into S) are alif_backward() on I_total, and dL/dW_rec is
 * syn_project_backward() of grad_I against the spikes delayed by T_R
 * (alif_delay_spikes). */
int alif_forward_recurrent(int64_t B, int64_t N, int64_t T, const float *I_ff, const float *W_rec_t,
                           const AlifNeuron *neurons, double dt_ms, double arp_ms,
                           const AlifState *init, float *I_total, uint32_t *spikes,
                           AlifState *ckpt, AlifState *final_state, void *stream);

/* Delayed spike raster (device, [B*N, ceil(T/32)] each): bit t of `delayed` =
 * bit t - D of `spikes` (0 for t < D); bits at t >= T are 0.  D >= 0; the two
 * arrays must not overlap. */
int alif_delay_spikes(int64_t B, int64_t N, int64_t T, int64_t D, const uint32_t *spikes,
                      uint32_t *delayed, void *stream);

/* ------------------------------------------ allocation-free backward   */

/* Largest B * N that alif_backward_noalloc() accepts. */
#define ALIF_NOALLOC_MAX_ROWS 65536

/* alif_backward() for callers that cannot allocate device memory when they
 * run the backward pass -- for example code working inside a memory budget
 * reserved in advance, or a host loop that must not call cudaMalloc/cudaFree
 * because those calls synchronise the device.  The paper has no counterpart;
 * this is a service of the library.
 * Same arguments, checks and results as alif_backward() without the workspace
 * (T = 0 included: zero parameter gradients, grad_init = grad_final); the
 * per-row partial sums live in a fixed array inside the library's device
 * memory (ALIF_NOALLOC_MAX_ROWS * 10 floats, 2.5 MiB, held on every GPU that
 * loads the library until the process exits).  Nothing is allocated: no
 * cudaMalloc, cudaFree or allocating library call is made.
 *   - B * N must be <= ALIF_NOALLOC_MAX_ROWS, else ALIF_ESHAPE (use
 *     alif_backward() with a workspace for larger batches).  Every argument
 *     check is made before any CUDA call.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  Host threads may make their first calls
 *     concurrently (they store the same address).
 *   - All calls share the one array and it keeps the last call's contents
 *     (each call overwrites every slot it reads, so nothing needs clearing);
 *     calls that overlap on the GPU -- on different streams, or from
 *     different host threads -- race on it.  Serialise them. */
int alif_backward_noalloc(int64_t B, int64_t N, int64_t T, const float *I,
                          const AlifNeuron *neurons, const AlifState *init,
                          const uint32_t *spikes, const AlifState *ckpt,
                          const float *grad_spikes, const float *grad_v, const float *grad_a,
                          const float *grad_final, float slope,
                          float *grad_I, float *grad_init, float *grad_params, void *stream);

/* ------------------------------------------- plain sequential comparator */

/* The standard model as a plain GPU kernel: one thread per row walking
 * t = 0..T-1 (Eqs 1-5 as written, FP32), no shared-memory staging and no
 * manual unrolling.  Same arguments and outputs as alif_forward, minus ckpt.
 * The comparator for the blocked kernel's speed-up (Section 4.1). */
int alif_forward_seq(int64_t B, int64_t N, int64_t T, const float *I,
                     const AlifNeuron *neurons, const AlifState *init,
                     uint32_t *spikes, float *v_trace, float *a_trace,
                     AlifState *final_state, void *stream);

/* Tuned sequential comparator: the same per-step recurrence and outputs as
 * alif_forward_seq, with the input staged for coalescing (a warp owns 32
 * rows and reads 32-step tiles as 128-byte row segments through shared
 * memory, the next tile's loads issued before the current one is walked).
 * It bounds what a well-implemented step-by-step kernel reaches on the same
 * inputs (Section 4.1 compares against the step-by-step model). */
int alif_forward_seq_staged(int64_t B, int64_t N, int64_t T, const float *I,
                            const AlifNeuron *neurons, const AlifState *init,
                            uint32_t *spikes, float *v_trace, float *a_trace,
                            AlifState *final_state, void *stream);

/* Plain sequential backward: one thread per row walking t = T-1..0 over the
 * FULL traces v_trace, a_trace saved by alif_forward_seq (what a step-by-step
 * implementation stores).  Outputs as alif_backward. */
int alif_backward_seq(int64_t B, int64_t N, int64_t T, const float *I,
                      const AlifNeuron *neurons, const AlifState *init,
                      const uint32_t *spikes, const float *v_trace, const float *a_trace,
                      const float *grad_spikes, const float *grad_v, const float *grad_a,
                      const float *grad_final, float slope,
                      float *grad_I, float *grad_init, float *grad_params,
                      void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------- synaptic projection  */

/* Splits FP32 weights W [N, Nin] (row-major) into two BF16 terms written with
 * row stride ldw (>= Nin): hi = bf16(W), lo = bf16(W - hi), both round-to-
 * nearest-even, so |W - hi - lo| <= 2^-16 |W| in the normal range; columns
 * Nin..ldw-1 are written as zero.  W, W_hi, W_lo are device pointers; W_hi and
 * W_lo hold N * ldw uint16 (BF16 bit patterns).  syn_project() needs ldw to be
 * a multiple of 64 (ALIF_PROJ_K_ALIGN). */
#define ALIF_PROJ_K_ALIGN 64
int syn_split_bf16(const float *W, int64_t N, int64_t Nin, int64_t ldw,
                   uint16_t *W_hi, uint16_t *W_lo, void *stream);

/* Synaptic projection, the feedforward input current of Eq 3 and Prop 3:
 *     I[b, i, t] = bias[i] + sum_j (W_hi[i, j] + W_lo[i, j]) S_in[b, j, t]
 * on the tcgen05 tensor cores (BF16 operands, FP32 accumulation; spikes are
 * exactly 0/1, so every product is exact and the result differs from the FP64
 * sum by at most sum_j |W[i,j]| S[b,j,t] (2^-16 + Nin 2^-24) plus one rounding).
 *   W_hi, W_lo  [N, ldw] BF16 from syn_split_bf16 (ldw % 64 == 0, 16-byte aligned)
 *   S_in        [B, Nin, ceil(T/32)] uint32 spike bits (bits at t >= T ignored)
 *   bias        [N] float or NULL (zero)
 *   I           [B, N, T] float output
 * Returns ALIF_ESHAPE for ldw % 64 != 0 or ldw < Nin, ALIF_EUNSUPPORTED when the
 * driver cannot encode the TMA tensor maps. */
int syn_project(int64_t B, int64_t Nin, int64_t N, int64_t T,
                const uint16_t *W_hi, const uint16_t *W_lo, int64_t ldw,
                const uint32_t *S_in, const float *bias, float *I, void *stream);

/* Workspace bytes syn_project_backward() needs: the per-batch-element partial
 * sums of grad_W / grad_bias (reduced in a fixed order) and the two BF16 terms
 * of W^T used for grad_Sin. */
size_t syn_project_backward_workspace_size(int64_t B, int64_t N, int64_t Nin);

/* Backward of syn_project (the feedforward term of Eq 3 / Prop 3):
 *   grad_W[i, j]     = sum_{b,t} grad_I[b, i, t] S_in[b, j, t]      [N, Nin]
 *   grad_bias[i]     = sum_{b,t} grad_I[b, i, t]                    [N]
 *   grad_Sin[b, j, t] = sum_i W[i, j] grad_I[b, i, t]               [B, Nin, T]
 * grad_W and grad_bias are event-driven over the spikes in FP32, deterministic.
 * grad_Sin runs on the tcgen05 tensor cores: W and grad_I are each split into
 * two BF16 terms (x = x_hi + x_lo up to 2^-16 |x|) and the products
 * W_hi G_hi + W_hi G_lo + W_lo G_hi are accumulated in FP32, so each output is
 * within sum_i |W_ij| |grad_I[b,i,t]| (3 2^-16 + (3N + 2) 2^-24) of the exact
 * sum.  W is the FP32 weight matrix [N, Nin] (needed only for grad_Sin).
 * Outputs may be NULL when not wanted.  workspace (256-byte aligned) must hold
 * syn_project_backward_workspace_size(B, N, Nin) bytes when any output is
 * requested.  ALIF_EUNSUPPORTED when the driver cannot encode the TMA tensor
 * maps. */
int syn_project_backward(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W,
                         const uint32_t *S_in, const float *grad_I, float *grad_W,
                         float *grad_Sin, float *grad_bias, void *workspace,
                         size_t workspace_bytes, void *stream);

/* Event-driven projection (the feedforward term of Eq 3 / Prop 3, as
 * syn_project): I[b,i,t] = bias_i + sum over the inputs j active at (b, t) of
 * W[i,j], visiting only the set bits.  The weights are the exact FP32 values
 * (no BF16 split); every sum runs in a fixed order (inputs ascending), so the
 * result is deterministic and within (k+1) 2^-24 (|bias_i| + sum_j |W_ij| S_j)
 * of the exact sum for k active inputs.
 *   W_t   [Nin, N] FP32, the transposed weights (syn_transpose_weights)
 *   S_in  [B, Nin, ceil(T/32)] spike bits; bias [N] or NULL; I [B, N, T] output
 * Needs ceil(Nin/1024)*1024*N < 2^31 (ALIF_EUNSUPPORTED otherwise).
 * Device pointers; asynchronous on `stream`. */
int syn_project_events(int64_t B, int64_t Nin, int64_t N, int64_t T, const float *W_t,
                       const uint32_t *S_in, const float *bias, float *I, void *stream);

/* W [N, Nin] -> W_t [Nin, N] (the layout syn_project_events reads). */
int syn_transpose_weights(const float *W, int64_t N, int64_t Nin, float *W_t, void *stream);

/* Spike bits [rows, ceil(T/32)] -> float 0/1 [rows, T] (Eq 1's S as a dense
 * tensor, e.g. for frameworks that differentiate through it). */
int alif_unpack_spikes(int64_t rows, int64_t T, const uint32_t *spikes, float *out, void *stream);

/* Spike train as float 0/1 [rows, T] -> bits [rows, ceil(T/32)] (bit t%32 of
 * word t/32 set where S != 0); the inverse of alif_unpack_spikes. */
int alif_pack_spikes(int64_t rows, int64_t T, const float *S, uint32_t *spikes, void *stream);

/* ---------------------------------- classification readout and loss    */

/* Leaky readout of the classification network (Supplementary,
 * "Classification"): an integrator without spike or reset,
 *     V_o[t] = beta_o V_o[t-1] + (1 - beta_o) I_o[t],  out[b,c] = sum_t V_o[t],
 *     I_o[b,c,t] = bias_c + sum_k W[c,k] S[b,k,t].
 * Computed as out[b,c] = sum_k W[c,k] counts[b,k] + bias_c w_sum with
 * counts[b,k] = sum_t w_t S[b,k,t] and w_t = 1 - beta_o^(T-t).
 *   spikes  [B, K, ceil(T/32)] bits of the last hidden layer
 *   W       [C, K] FP32; bias [C] or NULL
 *   w_t     [T] the weights 1 - beta_o^(T-t) (alif_readout_weights), w_sum their sum
 *   counts  [B, K] output (kept for the backward); out [B, C] output
 * Device pointers; asynchronous on `stream`. */
int alif_readout_forward(int64_t B, int64_t K, int64_t C, int64_t T, const uint32_t *spikes,
                         const float *W, const float *bias, const float *w_t, float w_sum,
                         float *counts, float *out, void *stream);

/* Host (all pointers HOST): the readout's time weights w_t = 1 - beta_o^(T-t),
 * t = 0..T-1, with beta_o = exp(-DT/tau) (the leaky readout's decay), computed in
 * FP64 and rounded once to FP32 into w_t[T]; *w_sum receives their FP64 sum. */
int alif_readout_weights(int64_t T, double dt_ms, double tau_ms, float *w_t, double *w_sum);

/* Backward of alif_readout_forward from grad_out [B, C]:
 *   grad_spikes [B, K, T] = w_t sum_c W[c,k] grad_out[b,c]   (NULL: not computed)
 *   grad_W [C, K] = sum_b grad_out[b,c] counts[b,k]; grad_bias [C] = w_sum sum_b grad_out[b,c]
 * Fixed summation order (deterministic). */
int alif_readout_backward(int64_t B, int64_t K, int64_t C, int64_t T, const float *W,
                          const float *w_t, float w_sum, const float *counts,
                          const float *grad_out, float *grad_spikes, float *grad_W,
                          float *grad_bias, void *stream);

/* Mean softmax cross-entropy over the batch: loss [1] = -(1/B) sum_b log
 * softmax(logits[b])[labels[b]], and grad_logits [B, C] (NULL: not computed).
 * labels [B] int32 in [0, C) (an invalid label gives a NaN loss); workspace
 * holds B floats. */
int alif_cross_entropy(int64_t B, int64_t C, const float *logits, const int32_t *labels,
                       float *loss, float *grad_logits, float *workspace, void *stream);

/* ------------------------------------------------- neuron-fit loss    */

/* Squared van Rossum distance between spike trains x and y (Supplementary,
 * "Neural fits"), per row, with the kernel k(t) = exp(-t / tau_R) on the DT grid:
 *     f[t] = e^{-DT/tau_R} f[t-1] + x[t] - y[t],   loss = (DT / tau_R) sum_t f[t]^2.
 *   x, y    [rows, ceil(T/32)] spike bits
 *   f_ckpt  [rows, ceil(T/chunk)] output: f entering each chunk (NULL if unused);
 *           chunk must be a positive multiple of 256
 *   loss    [rows] output, or NULL */
int alif_vanrossum_forward(int64_t rows, int64_t T, const uint32_t *x, const uint32_t *y,
                           double dt_ms, double tau_ms, int64_t chunk, float *f_ckpt,
                           float *loss, void *stream);

/* Gradient of that loss with respect to x on steps [t0, t1) (t0 a multiple of
 * 256), produced chunk by chunk from the last chunk to the first:
 *     grad[r, t - t0] = (2 DT / tau_R) g[t],  g[t] = f[t] + e^{-DT/tau_R} g[t+1].
 *   f_start [rows] f entering step t0 (from f_ckpt)
 *   g_carry [rows] in: g[t1] (0 for the last chunk); out: g[t0]
 *   grad    [rows, t1 - t0] output;  t1 - t0 <= 2^19 (ALIF_EUNSUPPORTED beyond) */
int alif_vanrossum_backward(int64_t rows, int64_t T, const uint32_t *x, const uint32_t *y,
                            double dt_ms, double tau_ms, int64_t t0, int64_t t1,
                            const float *f_start, float *g_carry, float *grad, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ALIF_H */
