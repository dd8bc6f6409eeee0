/*
 * ParRep oracle: a plain, slow, single-threaded CPU implementation of parallel
 * replica (ParRep) dynamics for stochastic reaction networks.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path: it is written independently from the paper's method.
 *
 * What it follows (Wang & Plechac, "Parallel replica dynamics method for
 * bistable stochastic reaction networks", arXiv 1705.06807):
 *   - Sec. II.A: reaction network, propensities lambda_j(x,c), stoichiometric
 *     vectors eta_j, generator Q (Eq. 1).
 *   - Sec. III.A, Algorithm 1: decorrelation, Fleming-Viot dephasing and the
 *     parallel step, with the clock T_s and the time integral I_s (here a
 *     time-weighted histogram, which gives I_s for every observable f).
 *   - Sec. IV and Appendix A: the path-space Fisher information matrix as the
 *     stationary expectation of sum_j lambda_j grad log lambda_j grad log
 *     lambda_j^T (Appendix A form), and the relative entropy rate
 *     E sum_j [lambda_j log(lambda_j/lambda'_j) - lambda_j + lambda'_j].
 *   - Sec. V.A (Table I): the Schloegl network.
 *   - Sec. V.B (Table IV with the switching rates F, G): the genetic switch,
 *     state (xi, m, p) stored as x[0] = 2 m + xi, x[1] = p, six channels and
 *     eight parameters (a, b, gamma, k0min, k0max, k1min, k1max, D), each
 *     differentiated independently.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   - Holding time tau = -log(u1)/a0 and the direct-method selection "first j
 *     with lambda_1+...+lambda_j > u2*a0" (Gillespie direct method, Sec. II.A).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *     seed, counter = (replica, step, cycle, stage tag).  binary64 mode: one
 *     call per step (words 0,1 -> u1 and 2,3 -> u2).  binary32 mode: a step
 *     needs two 23-bit uniforms, so one call serves two steps -- counter step
 *     field = step/2, words (0,1) for even and (2,3) for odd steps -- and in
 *     the dephasing, which only needs the choice uniform, four steps: counter
 *     step/4, word step%4.
 *   - Thresholds: STEPS mode = the paper's counts n_c, n_p; TIME mode = the
 *     decorrelation ends after t_corr units of consecutive in-W time, and the
 *     dephasing makes n_p = ceil(t_phase * a0(X~)) lockstep jumps of the
 *     embedded chain (the parallel step runs the embedded chain, so the
 *     dephasing targets the embedded chain's quasi-stationary law).
 *   - Fleming-Viot: an exited replica restarts from a uniformly chosen replica
 *     of its group (fv_group consecutive replicas) that is still in W after the
 *     same step; with no survivor in the group it restarts from X~.
 *   - The run stops at T_end: contributions are taken in (stage, step, replica)
 *     order and the one that crosses T_end is truncated.
 *   - FIM and RER are accumulated over [T_burn, T_end] and returned as sums
 *     (the caller divides by T_end - T_burn).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ERANGE (-5)

enum { OR_SCHLOGL = 1, OR_TOGGLE = 2, OR_GENETIC = 3 };
#define OR_NCH 6 /* most channels of a network */
#define OR_NPAR 8 /* most parameters of a network */
enum { OR_TIME = 0, OR_STEPS = 1 };
enum { OR_F64 = 0, OR_F32 = 1 };
enum { TAG_INIT = 0, TAG_DECORR = 1, TAG_DEPHASE = 2, TAG_FV = 3, TAG_PARALLEL = 4, TAG_SSA = 5 };

typedef struct {
    int32_t kind;        /* OR_SCHLOGL, OR_TOGGLE or OR_GENETIC */
    int32_t n_species;   /* 1 or 2 */
    double c[8];         /* rate constants (Schloegl c1..c4; toggle aU, nU, dU, aV, nV, dV;
                            genetic a, b, gamma, k0min, k0max, k1min, k1max, D) */
    double s[4];         /* Schloegl fixed factors: lambda_j = c_j * s_j * h_j(x) */
    int32_t hist_max[2]; /* states must stay in [0, hist_max] */
    int32_t n_regions;   /* region(x) = first i with a_i . x < b_i, else n_regions */
    int32_t reg_a[4][2];
    int64_t reg_b[4];
} or_network;

typedef struct {
    int32_t thresh_mode;
    int32_t precision;
    int64_t n_replicas;
    int32_t fv_group;
    int32_t x0_uniform_hi; /* > 0: x0 drawn uniformly from {0..hi} per species */
    double t_corr, t_phase;
    double T_end, T_burn;
    uint64_t seed;
    int32_t x0[2];
} or_config;

typedef struct {
    int64_t cycle;
    int32_t W;
    int32_t ended;       /* 1 if T_end was reached inside this cycle */
    int64_t decorr_steps;
    int64_t dephase_steps;
    int64_t n_star;      /* steps of the parallel stage (N*), 0 if not reached */
    int64_t k;           /* 0-based index K of the first exiting replica, -1 if none */
    int32_t x_tilde[2];  /* X~ after the cycle */
    double T_s;
} or_cycle;

typedef struct {
    double T_s;
    int64_t events_decorr;
    int64_t events_dephase;
    int64_t events_parallel_useful;
    int64_t cycles;
    int64_t escapes;
    int32_t x_final[2];
    int32_t x0[2];
    int32_t status;
    int32_t pad;
} or_result;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4 and Fig. 2).     */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t cyc, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = {a, b, cyc, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, w);
}

/* The four Philox words a step reads, and where u1 (and u2) sit in them:
 * binary64 mode: counter field `step`, words 0..3; binary32 mode: counter
 * field step/2, the pair (2*(step%2), 2*(step%2)+1).  `hi` is the counter
 * word above the step (replica, or the high step bits). */
static const uint32_t* step_words(uint64_t seed, uint32_t hi, uint64_t step, uint32_t cyc, uint32_t tag, int prec,
                                  uint32_t w[4])
{
    if (prec == 1) {
        uint64_t pair = step >> 1;
        draw(seed, hi, (uint32_t)pair, cyc, tag, w);
        return w + 2 * (int)(step & 1);
    }
    draw(seed, hi, (uint32_t)step, cyc, tag, w);
    return w;
}

/* Uniform in (0,1) from 52 random bits: (m + 1/2) 2^-52, exact in binary64. */
double or_u01_f64(uint32_t wa, uint32_t wb)
{
    uint64_t m = ((uint64_t)wa << 20) | (uint64_t)(wb >> 12);
    return ((double)m + 0.5) * 0x1p-52;
}

/* Uniform in (0,1) from 23 random bits: (m + 1/2) 2^-23, exact in binary32. */
float or_u01_f32(uint32_t w)
{
    uint32_t m = w >> 9;
    return ((float)m + 0.5f) * 0x1p-23f;
}

/* Uniform integer in {0..n-1}: floor(w * n / 2^32). */
static uint32_t pick(uint32_t w, uint32_t n)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Networks (Sec. II.A; Table I for Schloegl)                               */
/* ------------------------------------------------------------------------ */
static const int ETA[4][OR_NCH][2] = {
    {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{1, 0}, {-1, 0}, {1, 0}, {-1, 0}, {0, 0}, {0, 0}}, /* Schloegl: 2S->3S, 3S->2S, 0->S, S->0 */
    {{1, 0}, {0, 1}, {-1, 0}, {0, -1}, {0, 0}, {0, 0}}, /* toggle: make U, make V, lose U, lose V */
    /* genetic: transcription (m+1), mRNA decay (m-1), translation (p+1),
     * protein decay (p-1), activation (xi 0->1), deactivation (xi 1->0) */
    {{2, 0}, {-2, 0}, {0, 1}, {0, -1}, {1, 0}, {-1, 0}},
};

static int n_channels(const or_network* N) { return N->kind == OR_GENETIC ? 6 : 4; }

/* the genetic switch's Hill factor h = p^2/(p^2 + D^2) and switching rates
 * F = k0min + (k0max - k0min) h, G = k1max - (k1max - k1min) h */
static void genetic_rates(const double* c, double p, double* h, double* F, double* G)
{
    *h = p * p / (p * p + c[7] * c[7]);
    *F = c[3] + (c[4] - c[3]) * *h;
    *G = c[6] - (c[6] - c[5]) * *h;
}

/* propensities in binary64 (channels past n_channels are zero) */
static void props_f64(const or_network* N, const int32_t* x, double lam[OR_NCH])
{
    lam[4] = 0.0;
    lam[5] = 0.0;
    if (N->kind == OR_GENETIC) {
        double xi = (double)(x[0] & 1), m = (double)(x[0] >> 1), p = (double)x[1];
        double h, F, G;
        genetic_rates(N->c, p, &h, &F, &G);
        lam[0] = N->c[0] * xi;
        lam[1] = N->c[2] * m;
        lam[2] = (N->c[2] * N->c[1]) * m;
        lam[3] = p;
        lam[4] = F * (1.0 - xi);
        lam[5] = G * xi;
    } else if (N->kind == OR_SCHLOGL) {
        double xd = (double)x[0];
        double h1 = xd * (xd - 1.0);
        double h2 = h1 * (xd - 2.0);
        lam[0] = (N->c[0] * N->s[0]) * h1;
        lam[1] = (N->c[1] * N->s[1]) * h2;
        lam[2] = (N->c[2] * N->s[2]);
        lam[3] = (N->c[3] * N->s[3]) * xd;
    } else {
        double U = (double)x[0], V = (double)x[1];
        lam[0] = N->c[0] / (1.0 + pow(V, N->c[1]));
        lam[1] = N->c[3] / (1.0 + pow(U, N->c[4]));
        lam[2] = N->c[2] * U;
        lam[3] = N->c[5] * V;
    }
}

/* propensities in binary32 (the constants are rounded from binary64; the
 * toggle's production terms and the genetic switching rates are evaluated in
 * binary64 and rounded once) */
static void props_f32(const or_network* N, const int32_t* x, float lam[OR_NCH])
{
    lam[4] = 0.0f;
    lam[5] = 0.0f;
    if (N->kind == OR_GENETIC) {
        float xi = (float)(x[0] & 1), m = (float)(x[0] >> 1);
        double h, F, G;
        genetic_rates(N->c, (double)x[1], &h, &F, &G);
        lam[0] = (float)N->c[0] * xi;
        lam[1] = (float)N->c[2] * m;
        lam[2] = (float)(N->c[2] * N->c[1]) * m;
        lam[3] = (float)x[1];
        lam[4] = (float)F * (1.0f - xi);
        lam[5] = (float)G * xi;
    } else if (N->kind == OR_SCHLOGL) {
        float xf = (float)x[0];
        float h1 = xf * (xf - 1.0f);
        float h2 = h1 * (xf - 2.0f);
        lam[0] = (float)(N->c[0] * N->s[0]) * h1;
        lam[1] = (float)(N->c[1] * N->s[1]) * h2;
        lam[2] = (float)(N->c[2] * N->s[2]);
        lam[3] = (float)(N->c[3] * N->s[3]) * xf;
    } else {
        double U = (double)x[0], V = (double)x[1];
        lam[0] = (float)(N->c[0] / (1.0 + pow(V, N->c[1])));
        lam[1] = (float)(N->c[3] / (1.0 + pow(U, N->c[4])));
        lam[2] = (float)N->c[2] * (float)x[0];
        lam[3] = (float)N->c[5] * (float)x[1];
    }
}

/* Direct method selection over the first n channels: first j with
 * lambda_0 + ... + lambda_j > target (sums taken left to right).  If rounding
 * leaves no such j, the last channel with positive propensity. */
static int select_f64(const double lam[OR_NCH], int n, double target)
{
    double cum = lam[0];
    if (cum > target) return 0;
    for (int j = 1; j < n; ++j) {
        cum = cum + lam[j];
        if (cum > target) return j;
    }
    for (int j = n - 1; j >= 0; --j)
        if (lam[j] > 0.0) return j;
    return -1;
}

static int select_f32(const float lam[OR_NCH], int n, float target)
{
    float cum = lam[0];
    if (cum > target) return 0;
    for (int j = 1; j < n; ++j) {
        cum = cum + lam[j];
        if (cum > target) return j;
    }
    for (int j = n - 1; j >= 0; --j)
        if (lam[j] > 0.0f) return j;
    return -1;
}

/* total rate a0, summed left to right */
static double a0_f64(const double lam[OR_NCH], int n)
{
    double a = lam[0];
    for (int j = 1; j < n; ++j) a = a + lam[j];
    return a;
}

static float a0_f32(const float lam[OR_NCH], int n)
{
    float a = lam[0];
    for (int j = 1; j < n; ++j) a = a + lam[j];
    return a;
}

/* One SSA step at state x from the four Philox words: the holding time tau
 * (needs_tau) and the reaction J.  Returns J, or -1 if a0 <= 0. */
static int ssa_step(const or_network* N, int prec, const int32_t* x, const uint32_t* w, double* tau)
{
    const int n = n_channels(N);
    if (prec == OR_F64) {
        double lam[OR_NCH];
        props_f64(N, x, lam);
        double a0 = a0_f64(lam, n);
        if (!(a0 > 0.0)) return -1;
        double u1 = or_u01_f64(w[0], w[1]);
        double u2 = or_u01_f64(w[2], w[3]);
        *tau = -log(u1) / a0;
        return select_f64(lam, n, u2 * a0);
    } else {
        float lam[OR_NCH];
        props_f32(N, x, lam);
        float a0 = a0_f32(lam, n);
        if (!(a0 > 0.0f)) return -1;
        float u1 = or_u01_f32(w[0]);
        float u2 = or_u01_f32(w[1]);
        float t = -logf(u1) / a0;
        *tau = (double)t;
        return select_f32(lam, n, u2 * a0);
    }
}

static int region_of(const or_network* N, const int32_t* x)
{
    for (int i = 0; i < N->n_regions; ++i) {
        int64_t v = (int64_t)N->reg_a[i][0] * x[0];
        if (N->n_species > 1) v += (int64_t)N->reg_a[i][1] * x[1];
        if (v < N->reg_b[i]) return i;
    }
    return N->n_regions;
}

static int in_range(const or_network* N, const int32_t* x)
{
    for (int i = 0; i < N->n_species; ++i)
        if (x[i] < 0 || x[i] > N->hist_max[i]) return 0;
    return 1;
}

static int64_t bin_of(const or_network* N, const int32_t* x)
{
    if (N->n_species == 1) return x[0];
    return (int64_t)x[0] * (N->hist_max[1] + 1) + x[1];
}

static int n_params(const or_network* N) { return N->kind == OR_SCHLOGL ? 4 : (N->kind == OR_TOGGLE ? 6 : 8); }

/* d log lambda_j / d c_k for the network's rate constants (row j; only rows
 * of channels with positive propensity are used). */
static void grad_log(const or_network* N, const int32_t* x, double g[OR_NCH][OR_NPAR])
{
    memset(g, 0, sizeof(double) * OR_NCH * OR_NPAR);
    if (N->kind == OR_GENETIC) {
        const double* c = N->c;
        double p = (double)x[1], h, F, G;
        genetic_rates(c, p, &h, &F, &G);
        double dh = -2.0 * p * p * c[7] / ((p * p + c[7] * c[7]) * (p * p + c[7] * c[7]));
        g[0][0] = 1.0 / c[0];
        g[1][2] = 1.0 / c[2];
        g[2][1] = 1.0 / c[1];
        g[2][2] = 1.0 / c[2];
        if (F > 0.0) {
            g[4][3] = (1.0 - h) / F;
            g[4][4] = h / F;
            g[4][7] = (c[4] - c[3]) * dh / F;
        }
        if (G > 0.0) {
            g[5][5] = h / G;
            g[5][6] = (1.0 - h) / G;
            g[5][7] = -(c[6] - c[5]) * dh / G;
        }
    } else if (N->kind == OR_SCHLOGL) {
        for (int j = 0; j < 4; ++j) g[j][j] = 1.0 / N->c[j];
    } else {
        double U = (double)x[0], V = (double)x[1];
        g[0][0] = 1.0 / N->c[0];
        if (x[1] > 0) {
            double p = pow(V, N->c[1]);
            g[0][1] = -p * log(V) / (1.0 + p);
        }
        g[1][3] = 1.0 / N->c[3];
        if (x[0] > 0) {
            double p = pow(U, N->c[4]);
            g[1][4] = -p * log(U) / (1.0 + p);
        }
        g[2][2] = 1.0 / N->c[2];
        g[3][5] = 1.0 / N->c[5];
    }
}

/* ------------------------------------------------------------------------ */
/* Accumulation of contributions (Algorithm 1: T_s += tau, I_s += f(X) tau)  */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_network* N;
    const or_config* C;
    double T_s;
    int ended;
    double* hist_pre;
    double* hist_post;
    double* fim;
    const double* rer_cp;
    int n_rer;
    double* rer;
    int64_t* cnt_pre;  /* optional: holding times added to each bin (tests bound rounding per bin) */
    int64_t* cnt_post;
} acc_t;

static void add_fim_rer(acc_t* A, const int32_t* x, double w)
{
    const or_network* N = A->N;
    int l = n_params(N), nch = n_channels(N);
    double lam[OR_NCH], g[OR_NCH][OR_NPAR];
    props_f64(N, x, lam);
    if (A->fim) {
        grad_log(N, x, g);
        for (int j = 0; j < nch; ++j) {
            if (lam[j] == 0.0) continue;
            for (int a = 0; a < l; ++a)
                for (int b = 0; b < l; ++b)
                    A->fim[a * l + b] += w * lam[j] * g[j][a] * g[j][b];
        }
    }
    for (int k = 0; k < A->n_rer; ++k) {
        or_network Np = *N;
        for (int i = 0; i < l; ++i) Np.c[i] = A->rer_cp[k * l + i];
        double lp[OR_NCH];
        props_f64(&Np, x, lp);
        double h = 0.0;
        for (int j = 0; j < nch; ++j) {
            double t = lp[j] - lam[j];
            if (lam[j] > 0.0) t += lam[j] * log(lam[j] / lp[j]);
            h += t;
        }
        A->rer[k] += w * h;
    }
}

/* Adds the holding time tau spent at state x.  Returns 1 once T_end is hit. */
static int contribute(acc_t* A, const int32_t* x, double tau)
{
    if (A->ended) return 1;
    double rem = A->C->T_end - A->T_s;
    double t = tau;
    if (t >= rem) {
        t = rem;
        A->ended = 1;
    }
    double pre = 0.0, post = t;
    if (A->T_s < A->C->T_burn) {
        double room = A->C->T_burn - A->T_s;
        pre = t < room ? t : room;
        post = t - pre;
    }
    int64_t b = bin_of(A->N, x);
    if (A->hist_pre) A->hist_pre[b] += pre;
    if (A->hist_post) A->hist_post[b] += post;
    if (A->cnt_pre && pre > 0.0) A->cnt_pre[b] += 1;
    if (A->cnt_post && post > 0.0) A->cnt_post[b] += 1;
    if (post > 0.0) add_fim_rer(A, x, post);
    if (A->ended)
        A->T_s = A->C->T_end;
    else
        A->T_s += t;
    return A->ended;
}

/* ------------------------------------------------------------------------ */
/* Dephasing (Algorithm 1, dephasing step; Fleming-Viot respawn)            */
/* ------------------------------------------------------------------------ */
/* Number of lockstep jumps of the dephasing stage: n_p itself in STEPS mode;
 * in TIME mode ceil(t_phase * a0(X~)) with a0 in binary64, i.e. the number of
 * jumps X~ makes on average in t_phase time units. */
int64_t or_dephase_steps(const or_network* N, const or_config* C, const int32_t* x_tilde)
{
    if (C->thresh_mode == OR_STEPS) return (int64_t)C->t_phase;
    double lam[OR_NCH];
    props_f64(N, x_tilde, lam);
    double a0 = a0_f64(lam, n_channels(N));
    double n = ceil(C->t_phase * a0);
    if (!(n < 4294967295.0)) return OR_ERANGE;
    return (int64_t)n;
}

/* Runs the dephasing of one cycle from X~ in region W: n_p lockstep jumps of
 * the embedded chain by every replica, each followed by the Fleming-Viot
 * respawn of the replicas that left W.  xs: n_rep x 2 states out.  Returns
 * the number of lockstep steps, or a negative error. */
int64_t or_dephase(const or_network* N, const or_config* C, const int32_t* x_tilde, int32_t W,
                   uint32_t cycle, int32_t* xs, int64_t* events)
{
    int64_t R = C->n_replicas;
    int G = C->fv_group;
    if (R < 1 || G < 1) return OR_EINVAL;
    int64_t n_p = or_dephase_steps(N, C, x_tilde);
    if (n_p < 0) return n_p;
    int32_t* xn = (int32_t*)malloc(sizeof(int32_t) * 2 * R);
    char* exited = (char*)calloc(R, 1);
    int64_t* surv = (int64_t*)malloc(sizeof(int64_t) * G);
    if (!xn || !exited || !surv) return OR_ENOMEM;
    for (int64_t r = 0; r < R; ++r) {
        xs[2 * r] = x_tilde[0];
        xs[2 * r + 1] = x_tilde[1];
    }
    int64_t ev = 0, status = 0;
    for (int64_t i = 0; i < n_p; ++i) {
        /* every replica makes one jump of the embedded chain */
        for (int64_t r = 0; r < R; ++r) {
            uint32_t w[4];
            int J;
            if (C->precision == OR_F32) {
                /* the choice uniform only: word i%4 of counter (r, i/4, cycle, DEPHASE) */
                draw(C->seed, (uint32_t)r, (uint32_t)(i >> 2), cycle, TAG_DEPHASE, w);
                float lam[OR_NCH];
                props_f32(N, xs + 2 * r, lam);
                float a0 = a0_f32(lam, n_channels(N));
                J = a0 > 0.0f ? select_f32(lam, n_channels(N), or_u01_f32(w[i & 3]) * a0) : -1;
            } else {
                draw(C->seed, (uint32_t)r, (uint32_t)i, cycle, TAG_DEPHASE, w);
                double tau = 0.0;
                J = ssa_step(N, C->precision, xs + 2 * r, w, &tau);
            }
            if (J < 0) { status = OR_ERANGE; goto done; }
            ++ev;
            xn[2 * r] = xs[2 * r] + ETA[N->kind][J][0];
            xn[2 * r + 1] = xs[2 * r + 1] + ETA[N->kind][J][1];
            exited[r] = region_of(N, xn + 2 * r) != W;
            if (!exited[r] && !in_range(N, xn + 2 * r)) { status = OR_ERANGE; goto done; }
        }
        /* Fleming-Viot: exited replicas copy a uniformly chosen survivor of the group */
        for (int64_t g0 = 0; g0 < R; g0 += G) {
            int64_t g1 = g0 + G < R ? g0 + G : R;
            int ns = 0;
            for (int64_t r = g0; r < g1; ++r)
                if (!exited[r]) surv[ns++] = r;
            for (int64_t r = g0; r < g1; ++r) {
                if (!exited[r]) continue;
                if (ns > 0) {
                    uint32_t w[4];
                    draw(C->seed, (uint32_t)r, (uint32_t)i, cycle, TAG_FV, w);
                    int64_t s = surv[pick(w[0], (uint32_t)ns)];
                    xn[2 * r] = xn[2 * s];
                    xn[2 * r + 1] = xn[2 * s + 1];
                } else {
                    xn[2 * r] = x_tilde[0];
                    xn[2 * r + 1] = x_tilde[1];
                }
            }
        }
        memcpy(xs, xn, sizeof(int32_t) * 2 * R);
    }
done:
    free(xn); free(exited); free(surv);
    if (events) *events += ev;
    return status ? status : n_p;
}

/* ------------------------------------------------------------------------ */
/* Parallel step (Algorithm 1, parallel step)                               */
/* ------------------------------------------------------------------------ */
/* Runs the lockstep parallel step from the states xs (n_rep x 2) in region W.
 * With acc == NULL nothing is accumulated.  On exit: *n_star = N*, *k = K
 * (0-based), x_exit = X^K_{N*}.  Returns 0, 1 if T_end stopped it, or an
 * error.  max_steps bounds the stage (0 = unbounded). */
static int parallel_step(const or_network* N, const or_config* C, acc_t* A, int32_t* xs, int32_t W,
                         uint32_t cycle, int64_t max_steps, int64_t* n_star, int64_t* k_out,
                         int32_t* x_exit, int64_t* useful, double* tsum, double* hist)
{
    int64_t R = C->n_replicas;
    double* tau = (double*)malloc(sizeof(double) * R);
    int32_t* xn = (int32_t*)malloc(sizeof(int32_t) * 2 * R);
    char* ex = (char*)malloc(R);
    if (!tau || !xn || !ex) return OR_ENOMEM;
    int rc = 0;
    int64_t n = 0;
    *k_out = -1;
    for (;;) {
        if (max_steps > 0 && n >= max_steps) { rc = 2; break; }
        if (n >= 0xFFFFFFFFll) { rc = OR_ERANGE; break; }
        int64_t K = -1;
        for (int64_t r = 0; r < R; ++r) {
            uint32_t w[4];
            const uint32_t* ws = step_words(C->seed, (uint32_t)r, (uint64_t)n, cycle, TAG_PARALLEL, C->precision, w);
            int J = ssa_step(N, C->precision, xs + 2 * r, ws, &tau[r]);
            if (J < 0) { rc = OR_ERANGE; goto out; }
            xn[2 * r] = xs[2 * r] + ETA[N->kind][J][0];
            xn[2 * r + 1] = xs[2 * r + 1] + ETA[N->kind][J][1];
            ex[r] = region_of(N, xn + 2 * r) != W;
            if (ex[r] && K < 0) K = r;
        }
        int64_t last = K >= 0 ? K : R - 1;
        for (int64_t r = 0; r <= last; ++r) {
            if (A) {
                if (contribute(A, xs + 2 * r, tau[r])) { rc = 1; *n_star = n + 1; goto out; }
            }
            ++*useful;
            if (tsum) *tsum += tau[r];
            if (hist) hist[bin_of(N, xs + 2 * r)] += tau[r];
            if (!in_range(N, xn + 2 * r)) { rc = OR_ERANGE; goto out; }
        }
        ++n;
        if (K >= 0) {
            *n_star = n;
            *k_out = K;
            x_exit[0] = xn[2 * K];
            x_exit[1] = xn[2 * K + 1];
            break;
        }
        memcpy(xs, xn, sizeof(int32_t) * 2 * R);
    }
out:
    free(tau); free(xn); free(ex);
    return rc;
}

/* Escape-lemma helper: one parallel step from given states with no T_end.
 * tsum and hist (optional) receive the holding times of the contributions
 * (replicas r <= K at step N*, all replicas before).  Returns 0 on exit, 2 if
 * max_steps ran out. */
int or_parallel_from(const or_network* N, const or_config* C, int32_t* xs, int32_t W, uint32_t cycle,
                     int64_t max_steps, int64_t* n_star, int64_t* k, int32_t* x_exit, double* tsum,
                     double* hist)
{
    int64_t useful = 0;
    *n_star = 0;
    return parallel_step(N, C, NULL, xs, W, cycle, max_steps, n_star, k, x_exit, &useful, tsum, hist);
}

/* ------------------------------------------------------------------------ */
/* Full ParRep run (Algorithm 1 looped until T_s reaches T_end)             */
/* ------------------------------------------------------------------------ */
static int check_inputs(const or_network* N, const or_config* C)
{
    if (N->kind != OR_SCHLOGL && N->kind != OR_TOGGLE && N->kind != OR_GENETIC) return OR_EINVAL;
    if (N->n_species != (N->kind == OR_SCHLOGL ? 1 : 2)) return OR_EINVAL;
    if (N->n_regions < 1 || N->n_regions > 4) return OR_EINVAL;
    if (C->n_replicas < 1 || C->fv_group < 1) return OR_EINVAL;
    if (!(C->T_end >= 0.0) || !(C->T_burn >= 0.0)) return OR_EINVAL;
    if (!(C->t_corr >= 0.0) || !(C->t_phase >= 0.0)) return OR_EINVAL;
    return OR_OK;
}

void or_initial_state(const or_network* N, const or_config* C, int32_t x[2])
{
    x[0] = C->x0[0];
    x[1] = N->n_species > 1 ? C->x0[1] : 0;
    if (C->x0_uniform_hi > 0) {
        uint32_t w[4];
        draw(C->seed, 0, 0, 0, TAG_INIT, w);
        x[0] = (int32_t)pick(w[0], (uint32_t)C->x0_uniform_hi + 1u);
        if (N->n_species > 1) x[1] = (int32_t)pick(w[1], (uint32_t)C->x0_uniform_hi + 1u);
    }
}

/* or_parrep_run with, optionally, the number of holding times added to each
 * bin before and after T_burn (cnt_pre, cnt_post may be NULL). */
int or_parrep_run_counted(const or_network* N, const or_config* C, double* hist_pre, double* hist_post,
                          double* fim, const double* rer_cprime, int32_t n_rer, double* rer_out,
                          or_cycle* log, int64_t log_cap, int64_t* log_n, or_result* res,
                          int64_t* cnt_pre, int64_t* cnt_post)
{
    memset(res, 0, sizeof(*res));
    int rc = check_inputs(N, C);
    if (rc) { res->status = rc; return rc; }
    int64_t R = C->n_replicas;
    acc_t A = {N, C, 0.0, 0, hist_pre, hist_post, fim, rer_cprime, n_rer, rer_out, cnt_pre, cnt_post};
    int32_t xt[2];
    or_initial_state(N, C, xt);
    res->x0[0] = xt[0];
    res->x0[1] = xt[1];
    if (!in_range(N, xt)) { res->status = OR_EINVAL; return OR_EINVAL; }
    int32_t* xs = (int32_t*)malloc(sizeof(int32_t) * 2 * R);
    if (!xs) return OR_ENOMEM;
    if (log_n) *log_n = 0;
    int steps_mode = C->thresh_mode == OR_STEPS;
    uint32_t cycle = 0;
    int status = 0;
    if (C->T_end <= 0.0) A.ended = 1;
    while (!A.ended) {
        or_cycle rec;
        memset(&rec, 0, sizeof(rec));
        rec.cycle = cycle;
        rec.k = -1;
        /* ---- decorrelation ---- */
        int32_t W = region_of(N, xt);
        int64_t Nc = 0, step = 0;
        double inW = 0.0;
        for (;;) {
            if (steps_mode ? (Nc >= (int64_t)C->t_corr) : (inW >= C->t_corr)) break;
            uint32_t w[4];
            const uint64_t cs = C->precision == OR_F32 ? (uint64_t)step >> 1 : (uint64_t)step;
            draw(C->seed, (uint32_t)(cs >> 32), (uint32_t)cs, cycle, TAG_DECORR, w);
            const uint32_t* ws = C->precision == OR_F32 ? w + 2 * (int)(step & 1) : w;
            double tau = 0.0;
            int J = ssa_step(N, C->precision, xt, ws, &tau);
            if (J < 0) { status = OR_ERANGE; goto finish; }
            ++res->events_decorr;
            ++step;
            if (contribute(&A, xt, tau)) break;
            xt[0] += ETA[N->kind][J][0];
            xt[1] += ETA[N->kind][J][1];
            if (!in_range(N, xt)) { status = OR_ERANGE; goto finish; }
            int Wn = region_of(N, xt);
            if (Wn == W) {
                ++Nc;
                inW += tau;
            } else {
                Nc = 0;
                inW = 0.0;
                W = Wn;
            }
        }
        rec.W = W;
        rec.decorr_steps = step;
        if (A.ended) goto record;
        /* ---- dephasing ---- */
        {
            int64_t d = or_dephase(N, C, xt, W, cycle, xs, &res->events_dephase);
            if (d < 0) { status = (int)d; goto finish; }
            rec.dephase_steps = d;
        }
        /* ---- parallel step ---- */
        {
            int64_t n_star = 0, k = -1;
            int32_t xe[2] = {0, 0};
            int prc = parallel_step(N, C, &A, xs, W, cycle, 0, &n_star, &k, xe,
                                    &res->events_parallel_useful, NULL, NULL);
            if (prc < 0) { status = prc; goto finish; }
            rec.n_star = n_star;
            if (prc == 0) {
                rec.k = k;
                xt[0] = xe[0];
                xt[1] = xe[1];
                ++res->escapes;
            }
        }
    record:
        rec.ended = A.ended;
        rec.x_tilde[0] = xt[0];
        rec.x_tilde[1] = xt[1];
        rec.T_s = A.T_s;
        if (log && log_n && *log_n < log_cap) log[(*log_n)++] = rec;
        ++cycle;
        ++res->cycles;
    }
finish:
    free(xs);
    res->T_s = A.T_s;
    res->x_final[0] = xt[0];
    res->x_final[1] = xt[1];
    res->status = status;
    return status;
}

int or_parrep_run(const or_network* N, const or_config* C, double* hist_pre, double* hist_post,
                  double* fim, const double* rer_cprime, int32_t n_rer, double* rer_out,
                  or_cycle* log, int64_t log_cap, int64_t* log_n, or_result* res)
{
    return or_parrep_run_counted(N, C, hist_pre, hist_post, fim, rer_cprime, n_rer, rer_out, log, log_cap, log_n,
                                 res, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Plain Gillespie SSA (Sec. II.A) for n_traj independent trajectories       */
/* ------------------------------------------------------------------------ */
/* Trajectory t draws from counter (t, step low, step high, SSA).  hist is the
 * summed time-weighted histogram of all trajectories; events counts jumps. */
int or_ssa_run(const or_network* N, int32_t precision, int64_t n_traj, const int32_t* x0, double T_end,
               uint64_t seed, double* hist, int64_t* events, int32_t* x_final)
{
    *events = 0;
    for (int64_t t = 0; t < n_traj; ++t) {
        int32_t x[2] = {x0[0], N->n_species > 1 ? x0[1] : 0};
        double T = 0.0;
        uint64_t step = 0;
        if (!in_range(N, x)) return OR_EINVAL;
        while (T < T_end) {
            uint32_t w[4];
            const uint64_t cs = precision == OR_F32 ? step >> 1 : step;
            draw(seed, (uint32_t)t, (uint32_t)cs, (uint32_t)(cs >> 32), TAG_SSA, w);
            const uint32_t* ws = precision == OR_F32 ? w + 2 * (int)(step & 1) : w;
            double tau = 0.0;
            int J = ssa_step(N, precision, x, ws, &tau);
            if (J < 0) return OR_ERANGE;
            double rem = T_end - T;
            int64_t b = bin_of(N, x);
            if (tau >= rem) {
                hist[b] += rem;
                T = T_end;
                break;
            }
            hist[b] += tau;
            T += tau;
            x[0] += ETA[N->kind][J][0];
            x[1] += ETA[N->kind][J][1];
            ++*events;
            ++step;
            if (!in_range(N, x)) return OR_ERANGE;
        }
        if (x_final) {
            x_final[2 * t] = x[0];
            x_final[2 * t + 1] = x[1];
        }
    }
    return OR_OK;
}

/* Single trajectory SSA recording the first n_max (J, x after, tau) triples. */
int or_ssa_trace(const or_network* N, int32_t precision, const int32_t* x0, uint64_t seed, uint32_t traj,
                 int64_t n_max, int32_t* J_out, int32_t* x_out, double* tau_out)
{
    int32_t x[2] = {x0[0], N->n_species > 1 ? x0[1] : 0};
    for (int64_t s = 0; s < n_max; ++s) {
        uint32_t w[4];
        const uint64_t cs = precision == OR_F32 ? (uint64_t)s >> 1 : (uint64_t)s;
        draw(seed, traj, (uint32_t)cs, (uint32_t)(cs >> 32), TAG_SSA, w);
        const uint32_t* ws = precision == OR_F32 ? w + 2 * (int)(s & 1) : w;
        double tau = 0.0;
        int J = ssa_step(N, precision, x, ws, &tau);
        if (J < 0) return OR_ERANGE;
        x[0] += ETA[N->kind][J][0];
        x[1] += ETA[N->kind][J][1];
        J_out[s] = J;
        x_out[2 * s] = x[0];
        x_out[2 * s + 1] = x[1];
        tau_out[s] = tau;
    }
    return OR_OK;
}
