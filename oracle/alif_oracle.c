/*
 * ALIF oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential FP64 implementation of the *standard* step-by-step
 * adaptive leaky integrate-and-fire neuron of Taylor, King & Harper,
 * "Addressing the speed-accuracy simulation trade-off for adaptive spiking
 * neurons" (NeurIPS 2023), Section 2 "Standard ALIF model", Eqs 1-5, and its
 * surrogate-gradient BPTT with "detached" spikes (Supplementary, "Surrogate
 * gradient" and "Detaching gradients").
 *
 * The recurrent layer (Eq 3 with its recurrent term, transmission latency D =
 * T_R as Section 2 assumes) is stepped the same way, all neurons of a batch
 * element together (oracle_alif_forward_recurrent, at the end of the file).
 *
 * This file is the reference the CUDA path is checked against.  It is NOT the
 * blocked reformulation of Section 3: it walks time one step at a time exactly
 * as Eqs 1-5 are written.  Only tests/, the smoke check and the bench's CPU
 * baseline may load it; the product path never does.
 *
 * Conventions (readings of the paper, all also listed in the design notes):
 *  - Arrays are indexed k = 0..T-1 for the paper's t = 1..T.
 *  - The initial condition is the paper's state "at t = 0": V[0], S[0], a[0]
 *    and the refractory counter C[0] (steps since the last spike; use a value
 *    >= T_R, e.g. INT64_MAX, for "never spiked").  Rest = (0, 0, 0, never).
 *  - Eq 1 uses a strict comparison V > theta.
 *  - Eq 4: input enters iff C[t] >= T_R, with C[t] = t - (last spike time < t).
 *  - Eq 2 is generalised by a per-neuron input resistance R (effective input
 *    R * I[t]); R = 1 is the paper's normalised form.
 *  - Eq 5 is generalised by a per-neuron baseline theta0 (the paper fixes 1).
 *  - beta = exp(-DT / tau_mem), p = exp(-DT / tau_adapt)  (Supplementary,
 *    "Weight initialisation"); no clamping is applied.
 *  - T_R = ARP / DT rounded to the nearest integer; rejected when ARP / DT is
 *    further than 1e-9 (relative) from an integer or T_R < 1.
 *  - Gradient ("detached", the default): S[t-1] is a constant in the reset
 *    factor of Eq 2 and in the adaptation update of Eq 5; the ARP mask carries
 *    no gradient; dS/dV is replaced by a surrogate evaluated at u = V - theta
 *    (Supplementary, "Surrogate gradient"), and the gradient reaches theta as
 *    -dS/du.  "Attached" (Supplementary, "Detaching gradients"): the surrogate
 *    also carries the gradient of S[t] through the reset factor of V[t+1] and
 *    the update of a[t+1]; the ARP mask (an integer step count) still carries
 *    none.  Surrogates:
 *      0  fast sigmoid     1/(k|u|+1)^2 with slope k;
 *      1  multi-Gaussian   1.15 N(u|0, 0.5^2) - 0.15 N(u|3, 3^2) - 0.15 N(u|-3, 3^2),
 *         N(x|mu, s^2) the normal density, means and variances as printed;
 *      2  boxcar           0.5 where |u| <= 0.5, else 0.
 *
 * All state and arithmetic are double; float inputs are promoted exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_NEVER INT64_MAX

/* T_R from ARP and DT (Section 3.2: a block spans the ARP in time steps). */
int64_t oracle_tr(double dt, double arp)
{
    if (!(dt > 0.0) || !(arp > 0.0)) return -1;
    double q = arp / dt;
    double r = floor(q + 0.5);
    if (fabs(q - r) > 1e-9 * (q > 1.0 ? q : 1.0)) return -1;
    if (r < 1.0) return -1;
    return (int64_t)r;
}

typedef struct {
    int64_t B, N, T;
    const float *I;
    const double *tau_mem, *tau_adapt, *theta0, *d, *R;
    double dt;
    int64_t TR;
    const double *init_V;
    const uint8_t *init_S;
    const double *init_a;
    const int64_t *init_C;
    const int8_t *force;
    uint8_t *S;
    double *V, *a, *theta;
    uint8_t *mask;
    double *final_V;
    uint8_t *final_S;
    double *final_a;
    int64_t *final_C;
    /* backward */
    double slope;
    int surrogate;
    int attached;
    const double *gS, *gV, *ga;
    double *gI;
    double *g_tau_mem, *g_tau_adapt, *g_theta0, *g_d, *g_R, *g_V0, *g_a0;
    int64_t row_begin, row_end;
} oracle_job;

/* One neuron (row) forward: Eqs 1-5 one step at a time.  Writes the per-step
 * records into the row's slices of the optional output arrays. */
static void forward_row(const oracle_job *j, int64_t row,
                        uint8_t *S, double *V, double *a, double *th, uint8_t *m,
                        double *fV, uint8_t *fS, double *fa, int64_t *fC)
{
    const int64_t T = j->T;
    const int64_t i = row % j->N;
    const double beta = exp(-j->dt / j->tau_mem[i]);   /* Eq 2 decay */
    const double p = exp(-j->dt / j->tau_adapt[i]);    /* Eq 5 decay */
    const double th0 = j->theta0[i], d = j->d[i], R = j->R ? j->R[i] : 1.0;
    const float *I = j->I + row * T;
    const int8_t *force = j->force ? j->force + row * T : NULL;

    double V_prev = j->init_V ? j->init_V[row] : 0.0;
    double S_prev = j->init_S ? (double)j->init_S[row] : 0.0;
    double a_prev = j->init_a ? j->init_a[row] : 0.0;
    int64_t C_prev = j->init_C ? j->init_C[row] : ORACLE_NEVER;

    for (int64_t k = 0; k < T; ++k) {
        /* C[t]: steps following the last spike (Eq 4 prose). */
        int64_t C = (C_prev == ORACLE_NEVER) ? ORACLE_NEVER : C_prev + 1;
        /* Eq 5: adaptation and adaptive threshold. */
        double a_t = p * a_prev + S_prev;
        double theta = th0 + d * a_t;
        /* Eq 4: absolute refractory period gates the input current. */
        int admit = (C >= j->TR);
        double Iin = admit ? (double)I[k] : 0.0;
        /* Eq 2: membrane potential with reset by the previous spike. */
        double V_t = (beta * V_prev + (1.0 - beta) * R * Iin) * (1.0 - S_prev);
        /* Eq 1: spike when V exceeds the threshold (strict). */
        int s = (V_t > theta);
        if (force && force[k] >= 0) s = force[k];
        if (s) C = 0;

        if (S) S[k] = (uint8_t)s;
        if (V) V[k] = V_t;
        if (a) a[k] = a_t;
        if (th) th[k] = theta;
        if (m) m[k] = (uint8_t)admit;

        V_prev = V_t;
        S_prev = (double)s;
        a_prev = a_t;
        C_prev = C;
    }
    if (fV) *fV = V_prev;
    if (fS) *fS = (uint8_t)S_prev;
    if (fa) *fa = a_prev;
    if (fC) *fC = C_prev;
}

static void *forward_worker(void *arg)
{
    const oracle_job *j = (const oracle_job *)arg;
    const int64_t T = j->T;
    for (int64_t row = j->row_begin; row < j->row_end; ++row) {
        forward_row(j, row,
                    j->S ? j->S + row * T : NULL,
                    j->V ? j->V + row * T : NULL,
                    j->a ? j->a + row * T : NULL,
                    j->theta ? j->theta + row * T : NULL,
                    j->mask ? j->mask + row * T : NULL,
                    j->final_V ? j->final_V + row : NULL,
                    j->final_S ? j->final_S + row : NULL,
                    j->final_a ? j->final_a + row : NULL,
                    j->final_C ? j->final_C + row : NULL);
    }
    return NULL;
}

/* The surrogate dS/du at u = V - theta. */
static double normal_density(double x, double mu, double sd)
{
    const double z = (x - mu) / sd;
    const double two_pi = 6.283185307179586476925286766559;  /* 2 pi */
    return exp(-0.5 * z * z) / (sd * sqrt(two_pi));
}

static double surrogate(int kind, double slope, double u)
{
    if (kind == 1)
        return 1.15 * normal_density(u, 0.0, 0.5) - 0.15 * normal_density(u, 3.0, 3.0)
             - 0.15 * normal_density(u, -3.0, 3.0);
    if (kind == 2)
        return fabs(u) <= 0.5 ? 0.5 : 0.0;
    const double den = slope * fabs(u) + 1.0;
    return 1.0 / (den * den);
}

/* Reverse-mode pass for one row (surrogate gradient, detached or attached). */
static void backward_row(const oracle_job *j, int64_t row,
                         uint8_t *S, double *V, double *a, double *th, uint8_t *m)
{
    const int64_t T = j->T;
    const int64_t i = row % j->N;
    const double beta = exp(-j->dt / j->tau_mem[i]);
    const double p = exp(-j->dt / j->tau_adapt[i]);
    const double d = j->d[i], R = j->R ? j->R[i] : 1.0;
    const float *I = j->I + row * T;
    const double *gS = j->gS + row * T;
    const double *gV = j->gV ? j->gV + row * T : NULL;
    const double *ga = j->ga ? j->ga + row * T : NULL;
    double *gI = j->gI ? j->gI + row * T : NULL;

    forward_row(j, row, S, V, a, th, m, NULL, NULL, NULL, NULL);

    const double V0 = j->init_V ? j->init_V[row] : 0.0;
    const double S0 = j->init_S ? (double)j->init_S[row] : 0.0;
    const double a0 = j->init_a ? j->init_a[row] : 0.0;

    double GV_next = 0.0, Ga_next = 0.0;   /* dL/dV[t+1], dL/da[t+1] */
    double g_th0 = 0.0, g_d = 0.0, g_beta = 0.0, g_p = 0.0, g_R = 0.0;
    for (int64_t k = T - 1; k >= 0; --k) {
        const double u = V[k] - th[k];
        const double sg = surrogate(j->surrogate, j->slope, u);   /* surrogate dS/du */
        const double s_k = (double)S[k];
        const double s_km1 = (k > 0) ? (double)S[k - 1] : S0;
        const double V_km1 = (k > 0) ? V[k - 1] : V0;
        const double a_km1 = (k > 0) ? a[k - 1] : a0;
        const double Iin = m[k] ? (double)I[k] : 0.0;

        /* dL/dS[t]: the direct term; attached, also S[t]'s paths into
         * V[t+1] = (beta V[t] + (1 - beta) m R I[t+1]) (1 - S[t]) (Eq 2) and
         * a[t+1] = p a[t] + S[t] (Eq 5). */
        double GS = gS[k];
        if (j->attached && k + 1 < T) {
            const double Iin_next = m[k + 1] ? (double)I[k + 1] : 0.0;
            const double Vpre_next = beta * V[k] + (1.0 - beta) * R * Iin_next;
            GS += Ga_next - Vpre_next * GV_next;
        }
        /* dL/dV[t]: the spike term through the surrogate, the trace term and
         * the path into V[t+1] (reset factor with the value of S[t]). */
        double GV = sg * GS + (gV ? gV[k] : 0.0) + beta * (1.0 - s_k) * GV_next;
        /* dL/dtheta[t] = -dS/du * dL/dS; theta = theta0 + d a (Eq 5). */
        double Gth = -sg * GS;
        /* dL/da[t]: via theta, the trace, and a[t+1] = p a[t] + S[t]. */
        double Ga = d * Gth + (ga ? ga[k] : 0.0) + p * Ga_next;

        if (gI) gI[k] = (1.0 - beta) * R * (m[k] ? 1.0 : 0.0) * (1.0 - s_km1) * GV;
        g_th0 += Gth;
        g_d += a[k] * Gth;
        /* dV[t]/dbeta = (V[t-1] - R I[t]) (1 - S[t-1]). */
        g_beta += (1.0 - s_km1) * (V_km1 - R * Iin) * GV;
        /* da[t]/dp = a[t-1]. */
        g_p += a_km1 * Ga;
        /* dV[t]/dR = (1 - beta) I[t] (1 - S[t-1]). */
        g_R += (1.0 - beta) * Iin * (1.0 - s_km1) * GV;

        GV_next = GV;
        Ga_next = Ga;
    }
    const double tm = j->tau_mem[i], ta = j->tau_adapt[i];
    /* beta = exp(-DT/tau): dbeta/dtau = beta DT / tau^2 (same for p). */
    if (j->g_tau_mem) j->g_tau_mem[row] = g_beta * beta * j->dt / (tm * tm);
    if (j->g_tau_adapt) j->g_tau_adapt[row] = g_p * p * j->dt / (ta * ta);
    if (j->g_theta0) j->g_theta0[row] = g_th0;
    if (j->g_d) j->g_d[row] = g_d;
    if (j->g_R) j->g_R[row] = g_R;
    /* V[1] = (beta V[0] + ...)(1 - S[0]);  a[1] = p a[0] + S[0]. */
    if (j->g_V0) j->g_V0[row] = beta * (1.0 - S0) * GV_next;
    if (j->g_a0) j->g_a0[row] = p * Ga_next;
}

static void *backward_worker(void *arg)
{
    const oracle_job *j = (const oracle_job *)arg;
    const int64_t T = j->T;
    size_t n = (size_t)(T > 0 ? T : 1);
    uint8_t *S = (uint8_t *)malloc(n);
    uint8_t *m = (uint8_t *)malloc(n);
    double *V = (double *)malloc(n * sizeof(double));
    double *a = (double *)malloc(n * sizeof(double));
    double *th = (double *)malloc(n * sizeof(double));
    if (S && m && V && a && th)
        for (int64_t row = j->row_begin; row < j->row_end; ++row)
            backward_row(j, row, S, V, a, th, m);
    free(S); free(m); free(V); free(a); free(th);
    return NULL;
}

static int run_rows(oracle_job *base, int nthreads, void *(*fn)(void *))
{
    const int64_t rows = base->B * base->N;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > rows) nthreads = (int)(rows > 0 ? rows : 1);
    if (nthreads == 1) {
        base->row_begin = 0;
        base->row_end = rows;
        fn(base);
        return 0;
    }
    pthread_t tid[256];
    oracle_job jobs[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *base;
        jobs[t].row_begin = rows * t / nthreads;
        jobs[t].row_end = rows * (t + 1) / nthreads;
        if (pthread_create(&tid[t], NULL, fn, &jobs[t]) != 0) {
            fn(&jobs[t]);
            tid[t] = 0;
        } else {
            ++started;
        }
    }
    for (int t = 0; t < nthreads; ++t)
        if (tid[t]) pthread_join(tid[t], NULL);
    (void)started;
    return 0;
}

static int check_params(int64_t B, int64_t N, int64_t T, const double *tau_mem,
                        const double *tau_adapt)
{
    if (B < 0 || N < 0 || T < 0) return -2;
    for (int64_t i = 0; i < N; ++i)
        if (!(tau_mem[i] > 0.0) || !(tau_adapt[i] > 0.0)) return -3;
    return 0;
}

/* Forward simulation.  Returns 0, or <0 on invalid arguments. */
int oracle_alif_forward(int64_t B, int64_t N, int64_t T, const float *I,
                        const double *tau_mem, const double *tau_adapt,
                        const double *theta0, const double *d, const double *R,
                        double dt, double arp,
                        const double *init_V, const uint8_t *init_S,
                        const double *init_a, const int64_t *init_C,
                        const int8_t *force,
                        uint8_t *S, double *V, double *a, double *theta, uint8_t *mask,
                        double *final_V, uint8_t *final_S, double *final_a,
                        int64_t *final_C, int nthreads)
{
    int64_t TR = oracle_tr(dt, arp);
    if (TR < 1) return -1;
    int rc = check_params(B, N, T, tau_mem, tau_adapt);
    if (rc) return rc;
    oracle_job j;
    memset(&j, 0, sizeof j);
    j.B = B; j.N = N; j.T = T; j.I = I;
    j.tau_mem = tau_mem; j.tau_adapt = tau_adapt; j.theta0 = theta0; j.d = d; j.R = R;
    j.dt = dt; j.TR = TR;
    j.init_V = init_V; j.init_S = init_S; j.init_a = init_a; j.init_C = init_C;
    j.force = force;
    j.S = S; j.V = V; j.a = a; j.theta = theta; j.mask = mask;
    j.final_V = final_V; j.final_S = final_S; j.final_a = final_a; j.final_C = final_C;
    return run_rows(&j, nthreads, forward_worker);
}

/* Surrogate-gradient BPTT (attached = 0: detached, the paper's default).  Parameter gradients are per row (b, i);
 * the caller sums over the batch.  gS is required; gV, ga and all outputs are
 * optional.  `force` must equal the one given to the forward, if any. */
int oracle_alif_backward(int64_t B, int64_t N, int64_t T, const float *I,
                         const double *tau_mem, const double *tau_adapt,
                         const double *theta0, const double *d, const double *R,
                         double dt, double arp, double slope, int surrogate_kind,
                         int attached, const double *init_V, const uint8_t *init_S,
                         const double *init_a, const int64_t *init_C,
                         const int8_t *force,
                         const double *gS, const double *gV, const double *ga,
                         double *gI, double *g_tau_mem, double *g_tau_adapt,
                         double *g_theta0, double *g_d, double *g_R,
                         double *g_V0, double *g_a0, int nthreads)
{
    int64_t TR = oracle_tr(dt, arp);
    if (TR < 1) return -1;
    int rc = check_params(B, N, T, tau_mem, tau_adapt);
    if (rc) return rc;
    if (!gS) return -4;
    oracle_job j;
    memset(&j, 0, sizeof j);
    j.B = B; j.N = N; j.T = T; j.I = I;
    j.tau_mem = tau_mem; j.tau_adapt = tau_adapt; j.theta0 = theta0; j.d = d; j.R = R;
    j.dt = dt; j.TR = TR; j.slope = slope;
    if (surrogate_kind < 0 || surrogate_kind > 2) return -5;
    j.surrogate = surrogate_kind;
    j.attached = attached ? 1 : 0;
    j.init_V = init_V; j.init_S = init_S; j.init_a = init_a; j.init_C = init_C;
    j.force = force;
    j.gS = gS; j.gV = gV; j.ga = ga;
    j.gI = gI; j.g_tau_mem = g_tau_mem; j.g_tau_adapt = g_tau_adapt;
    j.g_theta0 = g_theta0; j.g_d = g_d; j.g_R = g_R; j.g_V0 = g_V0; j.g_a0 = g_a0;
    return run_rows(&j, nthreads, backward_worker);
}

/* ------------------------------------------------------------------------
 * Recurrent layer (Section 2, Eq 3 with its recurrent term; Section 2's
 * assumption that the recurrent transmission latency D equals the ARP, T_R):
 *     I_i[t] = I_ff_i[t] + sum_j W_rec[i][j] S_j[t - T_R]   (no spikes before t = 0),
 * where I_ff is the given feedforward current (bias + feedforward synapses).
 * Every neuron of a batch element is stepped together, one step at a time,
 * with the Eq 1-5 update of forward_row; batch elements are independent.
 * The recurrent sum runs over the presynaptic spikes in increasing j, in
 * double.  Outputs: S, V, a, theta, mask (optional, [B, N, T]) and the total
 * current I_total = I_ff + recurrent current (double, optional).
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t B, N, T, TR;
    const float *I_ff, *W_rec;
    const double *tau_mem, *tau_adapt, *theta0, *d, *R;
    double dt;
    uint8_t *S;
    double *V, *a, *theta, *I_total;
    uint8_t *mask;
    int64_t b_begin, b_end;
    int status;
} oracle_rec_job;

static void *recurrent_worker(void *arg)
{
    oracle_rec_job *j = (oracle_rec_job *)arg;
    const int64_t N = j->N, T = j->T, TR = j->TR;
    double *beta = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *V_prev = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *a_prev = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *S_prev = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    int64_t *C_prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t *pre = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    uint8_t *Sb = (uint8_t *)malloc((size_t)(N > 0 ? N : 1) * (size_t)(T > 0 ? T : 1));
    if (!beta || !p || !V_prev || !a_prev || !S_prev || !C_prev || !pre || !Sb) {
        j->status = -6;
        goto done;
    }
    for (int64_t i = 0; i < N; ++i) {
        beta[i] = exp(-j->dt / j->tau_mem[i]);   /* Eq 2 decay */
        p[i] = exp(-j->dt / j->tau_adapt[i]);    /* Eq 5 decay */
    }
    for (int64_t b = j->b_begin; b < j->b_end; ++b) {
        for (int64_t i = 0; i < N; ++i) {
            V_prev[i] = 0.0; a_prev[i] = 0.0; S_prev[i] = 0.0; C_prev[i] = ORACLE_NEVER;
        }
        for (int64_t k = 0; k < T; ++k) {
            /* presynaptic spikes T_R steps back (Section 2: D = T_R) */
            int64_t npre = 0;
            if (k >= TR)
                for (int64_t jn = 0; jn < N; ++jn)
                    if (Sb[jn * T + (k - TR)]) pre[npre++] = jn;
            for (int64_t i = 0; i < N; ++i) {
                const int64_t row = b * N + i;
                double Irec = 0.0;
                for (int64_t q = 0; q < npre; ++q) Irec += (double)j->W_rec[i * N + pre[q]];
                const double Itot = (double)j->I_ff[row * T + k] + Irec;  /* Eq 3 */
                int64_t C = (C_prev[i] == ORACLE_NEVER) ? ORACLE_NEVER : C_prev[i] + 1;
                double a_t = p[i] * a_prev[i] + S_prev[i];                 /* Eq 5 */
                double theta = j->theta0[i] + j->d[i] * a_t;
                int admit = (C >= TR);                                     /* Eq 4 */
                double Iin = admit ? Itot : 0.0;
                const double Ri = j->R ? j->R[i] : 1.0;
                double V_t = (beta[i] * V_prev[i] + (1.0 - beta[i]) * Ri * Iin) * (1.0 - S_prev[i]); /* Eq 2 */
                int s = (V_t > theta);                                     /* Eq 1 */
                if (s) C = 0;
                Sb[i * T + k] = (uint8_t)s;
                if (j->S) j->S[row * T + k] = (uint8_t)s;
                if (j->V) j->V[row * T + k] = V_t;
                if (j->a) j->a[row * T + k] = a_t;
                if (j->theta) j->theta[row * T + k] = theta;
                if (j->mask) j->mask[row * T + k] = (uint8_t)admit;
                if (j->I_total) j->I_total[row * T + k] = Itot;
                V_prev[i] = V_t;
                a_prev[i] = a_t;
                C_prev[i] = C;
            }
            /* S[t-1] of Eqs 2 and 5 for the next step: set after every neuron used the old one */
            for (int64_t i = 0; i < N; ++i) S_prev[i] = (double)Sb[i * T + k];
        }
    }
done:
    free(beta); free(p); free(V_prev); free(a_prev); free(S_prev); free(C_prev); free(pre); free(Sb);
    return NULL;
}

/* Recurrent forward.  W_rec: float [N, N] (row = postsynaptic neuron).  Returns 0, or
 * <0 on invalid arguments or when memory runs out (-6). */
int oracle_alif_forward_recurrent(int64_t B, int64_t N, int64_t T, const float *I_ff, const float *W_rec,
                                  const double *tau_mem, const double *tau_adapt,
                                  const double *theta0, const double *d, const double *R,
                                  double dt, double arp,
                                  uint8_t *S, double *V, double *a, double *theta, uint8_t *mask,
                                  double *I_total, int nthreads)
{
    int64_t TR = oracle_tr(dt, arp);
    if (TR < 1) return -1;
    int rc = check_params(B, N, T, tau_mem, tau_adapt);
    if (rc) return rc;
    if (!I_ff || !W_rec) return -4;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > B) nthreads = (int)(B > 0 ? B : 1);
    oracle_rec_job jobs[256];
    pthread_t tid[256];
    for (int t = 0; t < nthreads; ++t) {
        oracle_rec_job *jb = &jobs[t];
        memset(jb, 0, sizeof *jb);
        jb->B = B; jb->N = N; jb->T = T; jb->TR = TR;
        jb->I_ff = I_ff; jb->W_rec = W_rec;
        jb->tau_mem = tau_mem; jb->tau_adapt = tau_adapt; jb->theta0 = theta0; jb->d = d; jb->R = R;
        jb->dt = dt;
        jb->S = S; jb->V = V; jb->a = a; jb->theta = theta; jb->mask = mask; jb->I_total = I_total;
        jb->b_begin = B * t / nthreads;
        jb->b_end = B * (t + 1) / nthreads;
    }
    if (nthreads == 1) {
        recurrent_worker(&jobs[0]);
        return jobs[0].status;
    }
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&tid[t], NULL, recurrent_worker, &jobs[t]) != 0) {
            recurrent_worker(&jobs[t]);
            tid[t] = 0;
        }
    int st = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (tid[t]) pthread_join(tid[t], NULL);
        if (jobs[t].status) st = jobs[t].status;
    }
    return st;
}
