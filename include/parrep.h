/*
 * parrep.h -- C ABI of the GB300 (sm_103a) parallel replica (ParRep) library.
 *
 * The library runs the hot path of parallel replica dynamics for continuous
 * time Markov chains on bistable reaction networks (Wang & Plechac, arXiv
 * 1705.06807): Gillespie direct-method SSA replicas that go through the
 * decorrelation, Fleming-Viot dephasing and parallel steps of Algorithm 1,
 * the first-escape vote across replicas, and the time-weighted stationary
 * histogram from which the path-space Fisher information matrix and relative
 * entropy rates (Sec. IV, Appendix A) are contracted.
 *
 * Conventions for every entry point:
 *   - Return PARREP_OK (0) on success and a negative PARREP_E* code on error;
 *     parrep_last_error(h) then holds a one-line message (per handle).
 *   - Pointers passed in are only read during the call; the library copies
 *     what it keeps.  The library owns all device memory it allocates and
 *     frees it in parrep_destroy.
 *   - Output buffers may be host or device pointers (CUDA unified addressing
 *     decides); device outputs are written on the handle's stream and the
 *     call returns after the copy has completed.
 *   - One handle must not be used from two host threads at once.
 *   - Random numbers are Philox4x32-10 keyed by the 64-bit seed with the
 *     counter (replica, step, cycle, stage tag), so a run is reproducible
 *     from (network, options, T_end, seed) alone.
 *   - Time sums are kept in 64-bit fixed point with 2^-40 resolution (exact,
 *     order-independent addition); T_end must stay below 2^23.
 */
#ifndef PARREP_H
#define PARREP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PARREP_OK 0
#define PARREP_EINVAL (-1)   /* invalid argument (sizes, region spec, N < 1, ...) */
#define PARREP_ENOMEM (-2)   /* device allocation failed or the grid does not fit */
#define PARREP_ECUDA (-3)    /* a CUDA runtime call failed */
#define PARREP_ETIMEOUT (-4) /* a bounded device wait expired without progress */
#define PARREP_ERANGE (-5)   /* a state left [0, hist_max], or a counter overflowed */
#define PARREP_ESTATE (-6)   /* the call needs a completed run */

typedef struct parrep_s* parrep_t;

enum { PARREP_SCHLOGL = 1, PARREP_TOGGLE = 2, PARREP_GENETIC = 3 };
enum { PARREP_THRESH_TIME = 0, PARREP_THRESH_STEPS = 1 };
enum { PARREP_FP64 = 0, PARREP_FP32 = 1 };
/* Layout of the FP32 form's kernel: staged (each block's replica owner threads
 * walk the jump chains while helper warps draw the random numbers and account
 * the holding times -- the faster one for a few thousand replicas), direct
 * (one thread per replica -- faster from about 16384 replicas on), or auto
 * (direct from 16384 replicas on and for the genetic switch, which runs
 * direct only; staged otherwise).  Both give the same results bit for bit. */
enum { PARREP_F32_AUTO = 0, PARREP_F32_STAGED = 1, PARREP_F32_DIRECT = 2,
       /* batches and servers: each instance in the layout auto would give it
        * alone, in one kernel (for a single run the same as auto) */
       PARREP_F32_MIXED = 3 };

/* Reaction network (Sec. II.A).  Three kinds:
 *   PARREP_SCHLOGL (Table I, 1 species x):
 *     lambda_j = c[j] * s[j] * h_j(x),  h = (x(x-1), x(x-1)(x-2), 1, x),
 *     eta = (+1, -1, +1, -1).  s holds the fixed factors (1/2, 1/6, 1, 1 for
 *     combinatorial mass action; a/V, 1/V^2, bV, 1 for the volume form).
 *   PARREP_TOGGLE (2 species U = x[0], V = x[1]):
 *     lambda = (c0/(1+V^c1), c3/(1+U^c4), c2 U, c5 V),
 *     eta = (+U, +V, -U, -V).
 *   PARREP_GENETIC (Sec. V.B, Table IV; DNA state xi, mRNA m, protein p,
 *     stored as x[0] = 2 m + xi, x[1] = p), c = (a, b, gamma, k0min, k0max,
 *     k1min, k1max, D), h = p^2/(p^2 + D^2), F = k0min + (k0max - k0min) h,
 *     G = k1max - (k1max - k1min) h:
 *     lambda = (a xi, gamma m, gamma b m, p, F (1 - xi), G xi),
 *     eta = (m+1, m-1, p+1, p-1, xi 0->1, xi 1->0).  Binary64 form only:
 *     single runs, FIM/RER (eight parameters), batches, serving, parrep_uq,
 *     parrep_dephase, parrep_ssa and parrep_ssa_trace; the FP32 form and
 *     parrep_ssa_noalloc return EINVAL for this kind.
 * The sensitivity parameters are c (4 for Schloegl, 6 for the toggle, 8 for
 * the genetic switch). */
typedef struct {
    int32_t kind;          /* PARREP_SCHLOGL, PARREP_TOGGLE or PARREP_GENETIC */
    int32_t n_species;     /* 1 for Schloegl, 2 for the toggle and the genetic switch */
    double c[8];           /* rate constants */
    double s[4];           /* Schloegl fixed factors (ignored for the toggle) */
    int32_t x0[2];         /* initial state X~ = x_0 (Algorithm 1 set-up) */
    int32_t x0_uniform_hi; /* > 0: each species of x_0 drawn uniformly from {0..hi} */
    int32_t hist_max[2];   /* states must stay in [0, hist_max]; histogram bins */
} parrep_network;

/* Metastable sets (Sec. III.A): region(x) = the first i with
 * a[i][0]*x[0] + a[i][1]*x[1] < b[i], else n.  Integer arithmetic. */
typedef struct {
    int32_t n;          /* 1..4 tests, giving n+1 regions */
    int32_t a[4][2];
    int64_t b[4];
} parrep_regions;

typedef struct {
    int32_t thresh_mode;   /* PARREP_THRESH_TIME (default) or _STEPS */
    int32_t precision;     /* PARREP_FP64 (default) or PARREP_FP32 propensities */
    int32_t fv_group;      /* Fleming-Viot group size: 1,2,4,8,16 or 32 (default 32) */
    int32_t block_threads; /* CUDA block size, multiple of 32 up to 384 (0 = auto) */
    int32_t chunk_steps;   /* lockstep steps between escape votes (0 = auto: 2048 in the FP32
                              staged layout, else 256, halved down to 128 while a chunk would
                              hold more than 2^23 replica-steps) */
    int32_t debug_stall_barrier; /* fault injection: >= 0 makes block 0 leave at that
                                    grid barrier so the others time out; -1 = off */
    int32_t serial_stages; /* FP32 form: 1 runs the staged chunks without the owner /
                              helper overlap (same results; for tests), 0 = auto */
    int32_t max_blocks;    /* cap on the blocks of the run kernel (0 = auto: all groups of
                              replicas at once when the grid fits, else a full co-resident
                              grid); fewer blocks than groups run several groups per
                              block with the same results */
    int32_t f32_layout;    /* FP32 form: PARREP_F32_AUTO (default: direct from 16384
                              replicas on and for the genetic switch, else staged),
                              _STAGED or _DIRECT */
    double T_burn;         /* FIM / RER integrate over [T_burn, T_end] (default 0) */
    double wait_timeout_s; /* device wait limit without progress (default 10 s) */
    void* stream;          /* cudaStream_t to run on (NULL = legacy default stream) */
} parrep_options;

typedef struct {
    double T_s;                    /* simulated time reached (= T_end on success) */
    int64_t events_decorr;         /* decorrelation jumps (all count toward T_s) */
    int64_t events_dephase;        /* dephasing jumps (embedded chain, not in T_s) */
    int64_t events_parallel_useful;   /* parallel-step jumps whose time entered T_s */
    int64_t events_parallel_executed; /* parallel-step jumps simulated (first pass) */
    int64_t events_replay;         /* jumps re-simulated at the cut of a chunk */
    int64_t cycles;                /* ParRep cycles started */
    int64_t escapes;               /* parallel steps that ended by an escape */
    int64_t chunks;                /* escape votes */
    int64_t special_chunks;        /* votes that found an escape or a time cut */
    int32_t x0[2];                 /* the initial state used */
    int32_t x_final[2];            /* X~ at the end of the run */
    int32_t status;                /* PARREP_OK or the error of the run */
    int32_t grid_blocks;           /* blocks of the persistent launch */
    int32_t block_threads;
    int32_t chunk_steps;
    float kernel_ms;               /* device time of the run (CUDA events) */
    float pad;
    /* device cycles per phase, summed over blocks (thread 0 of each block):
     * decorrelation, dephasing, Philox draws, owner chains, accounting, grid
     * barriers, special-chunk work, vote reduction; then, inside block 0's
     * decorrelation, its draws, jump chain, holding times and ordered commit
     * (FP32 form; the FP64 form fills decorrelation, dephasing, barriers,
     * special and vote) */
    double phase_cycles[12];
} parrep_stats;

typedef struct {
    int64_t cycle;
    int32_t W;             /* region of the cycle's dephasing and parallel step */
    int32_t ended;         /* 1 if T_end was reached inside this cycle */
    int64_t decorr_steps;  /* decorrelation jumps of the cycle */
    int64_t dephase_steps; /* lockstep dephasing jumps n_p */
    int64_t n_star;        /* N*: lockstep steps of the parallel step (0: not reached) */
    int64_t k;             /* K, 0-based index of the first escaping replica; -1: none */
    int32_t x_tilde[2];    /* X~ after the cycle (the escape state X^K_{N*}) */
    double T_s;            /* clock at the end of the cycle */
} parrep_cycle;

/* Fills *opt with the defaults listed above. */
void parrep_default_options(parrep_options* opt);

/* Creates a ParRep engine for `net` with n_replicas = R replicas (Algorithm 1),
 * regions `reg`, and thresholds t_corr / t_phase.  TIME mode (default): the
 * decorrelation ends after t_corr time units of consecutive in-W time and the
 * dephasing makes ceil(t_phase * a0(X~)) lockstep jumps.  STEPS mode: t_corr
 * and t_phase are the paper's jump counts n_c and n_p (integers).
 * Allocates the device buffers; returns EINVAL, ENOMEM or ECUDA on failure. */
int parrep_create(const parrep_network* net, int64_t n_replicas, const parrep_regions* reg,
                  double t_corr, double t_phase, parrep_t* out);

/* Sets options (NULL restores the defaults).  Takes effect at the next run. */
int parrep_set_options(parrep_t h, const parrep_options* opt);

/* Runs Algorithm 1 from x_0 until the clock T_s reaches T_end (the crossing
 * holding time is truncated), in one persistent cooperative launch on the
 * handle's stream, and waits for it.  Resets all accumulators first.
 * Errors: EINVAL (T_end < 0 or >= 2^23, T_burn > T_end), ERANGE (a state left
 * [0, hist_max]), ETIMEOUT, ECUDA. */
int parrep_run(parrep_t h, double T_end, uint64_t seed);

/* Number of histogram bins: (hist_max[0]+1) * (hist_max[1]+1); bin of (U,V)
 * is U*(hist_max[1]+1)+V. */
int64_t parrep_n_bins(parrep_t h);

/* Time-weighted histogram of the run normalised by T_s: out[b] = (time spent
 * in bin b) / T_s -- the estimate of the stationary law pi (Sec. II.A ergodic
 * average).  len must equal parrep_n_bins. */
int parrep_histogram(parrep_t h, double* out, int64_t len);

/* Raw time sums per bin before and after T_burn (either pointer may be NULL). */
int parrep_histogram_raw(parrep_t h, double* pre, double* post, int64_t len);

/* Path-space FIM (Sec. IV; Appendix A form): the time average over
 * [T_burn, T_end] of sum_j lambda_j grad_c log lambda_j grad_c log lambda_j^T,
 * row-major l x l with l = 4 (Schloegl), 6 (toggle) or 8 (genetic switch,
 * its parameters taken independently); len = l*l. */
int parrep_fim(parrep_t h, double* out, int32_t len);

/* Relative entropy rates (Appendix A) H(P^c | P^{c'}) for n perturbed
 * parameter vectors c_prime (n x l, row-major): the time average over
 * [T_burn, T_end] of sum_j lambda_j log(lambda_j/lambda'_j) - lambda_j + lambda'_j. */
int parrep_rer(parrep_t h, const double* c_prime, int32_t n, double* out);

/* Run statistics (host pointer). */
int parrep_stats_get(parrep_t h, parrep_stats* out);

/* Per-cycle log of the last run (host pointer): up to cap records, *n_out set
 * to the number of cycles of the run (may exceed cap). */
int parrep_cycle_log(parrep_t h, parrep_cycle* out, int64_t cap, int64_t* n_out);

/* One dephasing stage (Algorithm 1) from x_tilde in region W for cycle index
 * `cycle` and `seed`, with the handle's replicas, thresholds and options;
 * out_states (host or device) receives n_replicas x 2 int32 states. */
int parrep_dephase(parrep_t h, const int32_t* x_tilde, int32_t W, uint32_t cycle, uint64_t seed,
                   int32_t* out_states);

void parrep_destroy(parrep_t h);

/* Message of the last error on h (or of the last failed parrep_create when
 * h is NULL).  Valid until the next call on h. */
const char* parrep_last_error(parrep_t h);

/* Plain Gillespie SSA (Sec. II.A) for n_traj independent trajectories, one
 * device thread each, from x0 to T_end.  Trajectory t draws from counter
 * (t, step low, step high, SSA tag).  hist_out (host or device, len = bins):
 * summed time-weighted histogram (time units); events_out (host, may be NULL):
 * total jumps; kernel_ms (host, may be NULL): device time.  stream may be NULL. */
int parrep_ssa(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end, uint64_t seed,
               double* hist_out, int64_t len, int64_t* events_out, float* kernel_ms, void* stream);

/* Plain SSA with a record of every jump, for trajectory-level checks (the
 * reaction index sequence and integer states of Sec. II.A's direct method).
 * The same counters and arithmetic as parrep_ssa: trajectory t starts at x0
 * and runs until T_end or until it has made max_steps jumps, whichever comes
 * first.  Outputs (host or device pointers, row-major per trajectory):
 *   reactions: n_traj x max_steps int32, the channel of each jump;
 *   states:    n_traj x max_steps x 2 int32, the state after each jump;
 *   holding:   n_traj x max_steps double (may be NULL), each holding time as
 *              the 2^-40 fixed-point value the library sums;
 *   n_jumps:   n_traj int64, the jumps made (entries beyond are not written);
 *   x_final:   n_traj x 2 int32, the state at the end.
 * Limits: n_traj * max_steps <= 2^28; x0_uniform_hi must be 0.
 * Returns PARREP_OK, EINVAL, ERANGE (a state left [0, hist_max]) or ECUDA. */
int parrep_ssa_trace(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end, uint64_t seed,
                     int64_t max_steps, int32_t* reactions, int32_t* states, double* holding, int64_t* n_jumps,
                     int32_t* x_final);

/* Limits of parrep_ssa_noalloc's fixed scratch. */
#define PARREP_SSA_NOALLOC_MAX_BINS 65536
#define PARREP_SSA_NOALLOC_MAX_SPECIES_STATES 4096

/* parrep_ssa for callers that cannot allocate device memory -- e.g. code
 * inside a framework that owns the whole device memory pool and forbids side
 * allocations, or a latency-sensitive loop in which cudaMalloc/cudaFree would
 * synchronise the device.  The paper has no counterpart: this is an interface
 * variant of the plain SSA above, with the same arguments, checks, results
 * and counters, except that hist_out (host or device, len = bins, time units)
 * is required, x0_uniform_hi must be 0 and no kernel time is reported.
 *   - The call waits for its stream (cudaStreamSynchronize) before it
 *     returns, like parrep_ssa, so it cannot be recorded in a stream capture;
 *     errors set parrep_last_error(NULL).
 *   - It calls no cudaMalloc/cudaFree and no allocating library routine.  Its
 *     scratch (fixed-point histogram, jump counter, status, toggle tables) is
 *     one file-scope device array of about 0.6 MB, which every GPU that loads
 *     the library holds until the process exits.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current.
 *   - Limits: at most PARREP_SSA_NOALLOC_MAX_BINS histogram bins and
 *     PARREP_SSA_NOALLOC_MAX_SPECIES_STATES states per species (hist_max+1);
 *     larger networks are rejected with PARREP_EINVAL.
 *   - All calls share the one array and clear it at the start; calls that
 *     overlap on the GPU (other streams, other host threads) race and must be
 *     serialised by the caller.
 * Returns PARREP_OK, PARREP_EINVAL, PARREP_ERANGE or PARREP_ECUDA. */
int parrep_ssa_noalloc(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end, uint64_t seed,
                       double* hist_out, int64_t len, int64_t* events_out, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent ParRep instances (different networks, system
 * sizes, replica counts, thresholds, T_end and seeds) in one persistent
 * cooperative launch.  Each instance is an ordinary handle made with
 * parrep_create / parrep_set_options; a batch groups n of them (it does not
 * own them) and runs Algorithm 1 for all at once.  After parrep_batch_run
 * every handle holds exactly the results parrep_run(h, T_end[i], seed[i])
 * would have given it (histograms, FIM, RER, statistics, cycle log -- read
 * with the single-run calls), bit for bit: an instance's arithmetic does not
 * depend on the blocks that run it.
 *
 * Scheduling: an instance's work is predicted from the block-cycles it took
 * in the batch's earlier runs, pooled: the parallel and decorrelation part
 * per unit of T_end, plus one dephasing of all replicas per cycle for a
 * cycle count two Poisson standard deviations above its measured mean
 * (before any run, an estimate from T_end * a0(x_0) plus one dephasing).  An instance whose
 * work exceeds the ideal makespan (total work / co-resident blocks) gets a
 * gang of blocks big enough to fit in it, capped by its groups of replicas;
 * gangs are placed longest-first on the grid, every block working through
 * its list of (instance, block index) in the schedule's start order.  A gang
 * smaller than an instance's replica groups takes several groups per block.
 * --------------------------------------------------------------------------- */
typedef struct parrep_batch_s* parrep_batch_t;

typedef struct {
    int32_t block_threads;      /* threads per block; 0 = chosen by the autotuner */
    int32_t replicas_per_block; /* FP32 staged layout: owner threads per block (32, 64, 128 or
                                   256); 0 = chosen by the autotuner.  FP64 form and FP32 direct
                                   layout: = block_threads */
    int32_t autotune;           /* 1 (default): the first run times candidate block shapes on a
                                   shortened copy of the batch (T_end scaled by tune_fraction)
                                   and keeps the fastest; 0: defaults (384 x 32 / 128) */
    int32_t use_graph;          /* 1 (default): capture the launch sequence (parameter upload,
                                   reset, batch kernel, read-back) in a CUDA graph and replay it
                                   while the shape stays the same */
    int32_t f32_layout;         /* FP32 form: PARREP_F32_AUTO (default) = _MIXED: each instance
                                   runs direct from 16384 replicas on and for the genetic switch,
                                   staged below; _STAGED (no genetic switch), _DIRECT */
    double tune_fraction;       /* default 0.05 */
    double wait_timeout_s;      /* device wait limit without progress anywhere (default 10 s) */
    void* stream;               /* cudaStream_t (NULL = legacy default stream) */
} parrep_batch_options;

typedef struct {
    int32_t block_threads, replicas_per_block;
    int32_t grid_blocks;        /* co-resident blocks of the launch */
    int32_t n_items;            /* (instance, block) pairs of the schedule */
    int32_t graph;              /* 1: the last run replayed a CUDA graph */
    int32_t tuned_trials;       /* shapes timed by the autotuner so far */
    int32_t f32_layout;         /* the launch's FP32 layout (PARREP_F32_STAGED, _DIRECT or
                                   _MIXED; 0 in the FP64 form) */
    int32_t pad;
    float kernel_ms;            /* last run: device time of the launch sequence (parameter
                                   upload, reset, batch kernel, read-back) */
    float tune_ms;              /* wall time spent autotuning */
    double est_makespan;        /* the schedule's makespan in its work units (block-cycles
                                   measured in the previous run, else estimated events) */
    double est_balance;         /* total work / (grid_blocks x makespan) */
} parrep_batch_info;

void parrep_batch_default_options(parrep_batch_options* opt);

/* Groups n handles (all with the same precision option) into a batch.
 * The handles must outlive the batch and must not run on their own while
 * the batch runs.  Errors: EINVAL (n < 1, null or repeated handle, mixed
 * precision), ENOMEM, ECUDA. */
int parrep_batch_create(const parrep_t* instances, int32_t n, const parrep_batch_options* opt,
                        parrep_batch_t* out);

/* Runs every instance i to T_end[i] with seed[i] (host arrays of n) in one
 * launch and waits.  Returns PARREP_OK when all instances succeeded, else
 * the first instance's error code in batch order (see parrep_batch_status).
 * Argument errors (T_end out of range, ...) are reported before anything
 * runs. */
int parrep_batch_run(parrep_batch_t b, const double* T_end, const uint64_t* seed);

/* Per-instance status of the last run (host array of n). */
int parrep_batch_status(parrep_batch_t b, int32_t* status_out);

int parrep_batch_info_get(parrep_batch_t b, parrep_batch_info* out);

void parrep_batch_destroy(parrep_batch_t b);

/* Message of the last error on b (or of the last failed parrep_batch_create
 * when b is NULL). */
const char* parrep_batch_last_error(parrep_batch_t b);

/* ---------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  One persistent serve
 * kernel polls a ring of requests (published through a host-mapped counter);
 * a block that claims
 * a newly published request leads it, and at every cycle start (Algorithm 1)
 * the request's leader recruits idle blocks into its gang, so requests that
 * arrive while others run start at once on free blocks and their work
 * overlaps on the device; a gang leaves an eighth of the blocks, and one
 * block for every published request not yet claimed, idle for those.  Requests are admitted by device memory: their
 * buffers (replica states, histograms, tables) come from one arena allocated
 * at parrep_server_create, first fit, in arrival order.  The replica state
 * stays in the arena from admission to the result.  The last block of a
 * request's gang writes its outputs (histogram normalised by T_s, FIM and
 * RER over [T_burn, T_s], statistics) and flags it done.  A request's
 * results depend only on the request: the same alone and in any mix, and the
 * same as parrep_run of a handle with the same network, options and seed.
 * A background host thread admits requests, (re)launches the serve kernel
 * when requests wait and it has left, and collects completions.
 * --------------------------------------------------------------------------- */
typedef struct parrep_server_s* parrep_server_t;

typedef struct {
    int32_t precision;          /* PARREP_FP64 or PARREP_FP32, for every request */
    int32_t block_threads;      /* 0 = 384 (FP32) / 128 (FP64) */
    int32_t replicas_per_block; /* FP32 form: owner threads per block (32..256), 0 = 32 */
    int32_t ring;               /* request slots (default 4096); a slot is reused after its result is read */
    int32_t f32_layout;         /* FP32 form: PARREP_F32_MIXED (default) / _AUTO (each request in
                                   the layout auto gives it: direct from 16384 replicas on and
                                   for genetic switches, staged below), _STAGED or _DIRECT */
    int64_t arena_bytes;        /* device memory for admitted requests (default 4 GiB) */
    int64_t log_cap;            /* cycle-log records kept per request (default 4096) */
    double idle_exit_s;         /* the serve kernel ends after the server has had nothing to do this
                                   long (default 0.05 s); the next request relaunches it */
    double wait_timeout_s;      /* device wait limit without progress (default 10 s) */
} parrep_server_options;

typedef struct {
    parrep_network net;
    parrep_regions regions;
    int64_t n_replicas;
    double t_corr, t_phase;     /* as in parrep_create */
    double T_end, T_burn;       /* as in parrep_run / parrep_options */
    uint64_t seed;
    int32_t thresh_mode;        /* PARREP_THRESH_TIME or PARREP_THRESH_STEPS */
    int32_t fv_group;           /* 0 = 32 */
    int32_t chunk_steps;        /* 0 = default */
    int32_t n_cprime;           /* perturbed parameter vectors for the RER (0..8) */
    const double* c_prime;      /* n_cprime x l (l = 4 Schloegl, 6 toggle, 8 genetic), copied at submit */
} parrep_request;

enum { PARREP_REQ_QUEUED = 0, PARREP_REQ_RUNNING = 1, PARREP_REQ_DONE = 2 };

typedef struct {
    int64_t submitted, admitted, completed, released;
    int64_t launches;           /* serve-kernel launches so far */
    int64_t queued, running;    /* requests waiting for admission / admitted and not done */
    int64_t arena_bytes, arena_used;
    int32_t grid_blocks, block_threads;
} parrep_server_stats;

void parrep_server_default_options(parrep_server_options* opt);

/* Allocates the arena, the ring and the serve kernel's state and starts the
 * host thread.  Errors: EINVAL, ENOMEM, ECUDA. */
int parrep_server_create(const parrep_server_options* opt, parrep_server_t* out);

/* Checks and copies a request and queues it; returns at once with its id.
 * EINVAL for an invalid request or one that can never fit the arena. */
int parrep_server_submit(parrep_server_t s, const parrep_request* req, int64_t* id);

/* State of a request: PARREP_REQ_QUEUED, _RUNNING or _DONE. */
int parrep_server_poll(parrep_server_t s, int64_t id, int32_t* state);

/* Waits until the request is done; ETIMEOUT after timeout_s (the request
 * stays in the server). */
int parrep_server_wait(parrep_server_t s, int64_t id, double timeout_s);

/* After parrep_server_wait: copies the results to host buffers (any may be
 * NULL) and releases the request's memory and slot.  hist: len = bins;
 * fim: l*l values; rer: n_cprime values; latency_s: submit to completion as
 * seen by the host thread.  Returns the request's own status (PARREP_OK, or
 * ERANGE / ETIMEOUT of its run); ESTATE if it is not done. */
int parrep_server_result(parrep_server_t s, int64_t id, parrep_stats* stats, double* hist, int64_t len,
                         double* fim, double* rer, double* latency_s);

int parrep_server_stats_get(parrep_server_t s, parrep_server_stats* out);

/* Stops accepting work, lets running requests finish, and frees everything. */
void parrep_server_destroy(parrep_server_t s);

const char* parrep_server_last_error(parrep_server_t s);

/* Stationary uncertainty quantification over independent runs (Sec. IV.B,
 * and the appendix that derives the stationary information bound
 * S_{f,v}(pi) <= sqrt(tau(f)) sqrt(v^T I_H v)).  The samples are n handles
 * that each completed a run of the same network shape (kind, hist_max) and
 * the same window [T_burn, T_end] (equal T_end - T_burn); their seeds should
 * differ.  With Y_k the integral of f over the window of sample k (from its
 * post-burn time sums) and w = T_end - T_burn:
 *   iaf            = sum_k (Y_k - Ybar)^2 / (w (n - 1))   (the IAF estimator)
 *   mean_f         = Ybar / w                             (estimate of pi(f))
 *   fim            = the mean over samples of the per-sample FIM (parrep_fim)
 *   fim_half_width = 1.96 sd / sqrt(n) per entry (normal 95% half widths)
 *   bound[k]       = sqrt(iaf) sqrt(fim[k][k])            (v = e_k)
 * Everything is computed on the device in binary64 in a fixed order (the
 * result does not depend on scheduling). */
typedef struct {
    int32_t n_samples;
    int32_t n_params;          /* l = 4 (Schloegl), 6 (toggle) or 8 (genetic switch) */
    double window;             /* w = T_end - T_burn */
    double iaf;
    double mean_f;
    double fim[64];            /* row-major l x l */
    double fim_half_width[64];
    double bound[8];
} parrep_uq_result;

/* handles: n >= 2 handles (host array).  f: one value per histogram bin
 * (host or device, len = parrep_n_bins).  dirs / n_dirs / dir_bounds
 * (optional, host or device): n_dirs directions v (n_dirs x l, row-major)
 * and their bounds sqrt(iaf) sqrt(v^T fim v).  Y_out (optional, host or
 * device, n values): the window integrals Y_k.  out: host pointer.
 * Errors: EINVAL (n < 2, a NULL handle or the same handle twice, mismatched
 * shapes or windows, len, empty window), ESTATE (a handle without a
 * completed run), ECUDA.  Runs on the first handle's stream. */
int parrep_uq(const parrep_t* handles, int32_t n, const double* f, int64_t len, const double* dirs, int32_t n_dirs,
              double* dir_bounds, double* Y_out, parrep_uq_result* out);

/* Device Philox4x32-10 of n counters (ctr: n x 4, key: n x 2, out: n x 4
 * uint32, all host pointers) -- exposes the generator the kernels use. */
int parrep_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out);

#ifdef __cplusplus
}
#endif

#endif /* PARREP_H */
