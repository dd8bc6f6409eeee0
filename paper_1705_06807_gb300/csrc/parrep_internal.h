// Internal declarations shared by the CUDA kernels and the host side of the
// C ABI.  Not part of the public interface (that is include/parrep.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "parrep.h"

namespace parrep {

// Time sums are unsigned 64-bit fixed point with 2^-40 resolution: a holding
// time tau is stored as round(tau * 2^40).  Addition is exact and
// order-independent, so sums do not depend on the order in which replicas
// finish, and a contribution added by a first pass can be taken back exactly.
constexpr int kQBits = 40;
constexpr double kQScale = 1099511627776.0;  // 2^40
constexpr double kQInv = 1.0 / 1099511627776.0;
constexpr double kTEndLimit = 8388608.0;     // 2^23: keeps every sum below 2^63

// Stage tags in the last word of the Philox counter.
enum Tag : uint32_t { kTagInit = 0, kTagDecorr = 1, kTagDephase = 2, kTagFV = 3, kTagParallel = 4, kTagSSA = 5 };

constexpr unsigned long long kNone = ~0ull;

// Largest block of the run kernels (their register budget is set for it).
constexpr int kMaxThreads = 384;
// binary32 direct form: threads per block and blocks per SM it is built for
constexpr int kDirectThreads = 256;
constexpr int kDirectMinBlocks = 3;

// Network as the kernels see it (Sec. II.A).  Schloegl: lambda_j = A[j] h_j(x)
// with A[j] = c_j s_j.  Toggle: production rates come from host-built tables
// indexed by the repressor count, degradation is d * count.
struct NetDev {
    int kind, nsp;
    int hist_max0, hist_max1, ystride, nbins;
    int nreg;
    int ra0[4], ra1[4];
    long long rb[4];
    // one species: region i is the interval [wlo[i], whi[i]] of [0, hist_max]
    // (an intersection of half-lines); empty when wlo > whi
    int wlo[5], whi[5];
    double A[4];
    float Af[4];
    double dU, dV;
    float dUf, dVf;
    const double* prodU_d;  // production of U as a function of V: c0/(1+V^c1)
    const double* prodV_d;  // production of V as a function of U: c3/(1+U^c4)
    const float* prodU_f;
    const float* prodV_f;
};

struct CycleRecDev {
    long long cycle;
    int W, ended;
    long long decorr_steps, dephase_steps, n_star, k;
    int xt0, xt1;
    unsigned long long Ts;
};

// Mutable state of one run, in global memory, zeroed before the launch.
struct RunCtl {
    unsigned int bar_count, bar_gen;
    unsigned long long progress;
    int status, done;
    int xt0, xt1, W, burn_done;
    unsigned int cycle, pad0;
    unsigned long long Ts;
    long long np;
    // first-pass vote of each chunk, rotated over three slots
    unsigned long long minkey[3], oobkey[3], chunksum[3], chunkev[3];
    unsigned long long inc_sum[3], inc_ev[3];
    // cut positions of a special chunk
    unsigned long long posT, partT, posB, partB;
    int xe0, xe1;
    // batches: the gang's current block count, and what a block that joins
    // at a cycle start needs to continue in step with the others
    int nblk;
    unsigned exited;  // blocks of the gang that have left the run
    unsigned long long chunk_c, est_q, est_ev;
    // statistics
    unsigned long long ev_decorr, ev_dephase, ev_par_exec, ev_useful, ev_replay;
    unsigned long long escapes, chunks, special, cycles;
    long long log_n;
    int x00, x01;
    // per-phase device cycles summed over blocks (thread 0 of each block):
    // decorrelation, dephasing, draw (P), owner chain (C), accounting (A),
    // grid barriers, special-chunk work, first-pass vote reduction
    unsigned long long phase_cycles[12];
};

// Shared state of a batch launch: instances not yet finished, the idle
// blocks (a bit each) and one mailbox per block through which an instance
// hands an idle block its place in the gang.
struct BatchDev {
    int* remaining;
    unsigned* idle;   // [ceil(grid / 32)]
    int4* mail;       // [grid]: (instance, block index in the gang, barrier generation, valid)
    // serving: requests published (host-mapped) and claimed; a gang recruits
    // only while no published request waits for a block (nullptr: batches)
    const unsigned long long* tail;
    const unsigned long long* head;
    int reserve;      // idle blocks a gang leaves unclaimed (room for new requests)
    int pad;
};

// Kernel forms: binary64 (one thread per replica), binary32 staged (owner
// threads + helper warps per block, for few replicas per SM), binary32 direct
// (one thread per replica at high occupancy, for many replicas).
// FP32 staged layout: steps staged per sub-chunk (96 with one owner warp a
// block, 32 with more), and the entries of the Schloegl threshold table
// beyond each end of [0, hist_max] (a speculative owner pass runs at most one
// sub-chunk past an exit, reading one state further on each side).
constexpr int kStagedB = 96;
inline int staged_sub_chunk(int RB) { return RB == 32 ? kStagedB : 32; }
constexpr int kThrPad = kStagedB + 2;

enum Form { kFormF64 = 0, kFormF32Staged = 1, kFormF32Direct = 2,
            // batch and serve kernels only: every instance runs its own
            // binary32 layout (RunParams::form, staged or direct)
            kFormF32Mixed = 3 };

struct RunParams {
    NetDev net;
    int prec, thresh;
    int form;      // Form of the kernel that runs this instance
    int R, G, S;
    int use_smem_hist;
    // block layout: the first RB threads of a block own replicas (RB = blockDim.x
    // in the FP64 form); the FP32 form stages B steps at a time through shared
    // memory (byte offsets of its arrays in the dynamic shared memory below)
    int RB, log2RB, B;
    int off_tab, off_buf, off_trace, off_live, off_nvalid;
    int off_limbs, off_inv, off_rng, off_decp;
    int off_thr;    // FP32 Schloegl: per-state choice thresholds (-1: none)
    int pipelined;  // FP32: owner warps and helper warps overlap (three draw slots, two trace slots)
    unsigned long long q_tcorr;
    long long n_c;
    double t_phase;
    long long n_p;
    unsigned long long q_Tend, q_Tburn;
    unsigned long long seed;
    int x00, x01, x0_hi;
    int nblk;      // blocks serving this instance (the grid, or a gang of a batch)
    int2* xs;      // [R] replica state between phases
    int2* xk;      // [R] replica state at the start of the current chunk
    int2* xe;      // [R] state a replica escaped to in the current chunk
    BatchDev batch;  // batches only (batch.remaining == nullptr otherwise)
    int inst;        // index of the instance in its batch
    RunCtl* ctl;
    unsigned long long* progress;  // heartbeat of the barriers: the run's own, or a whole batch's
    unsigned long long* hist_pre;
    unsigned long long* hist_post;
    unsigned long long* step_sum;  // S entries
    unsigned long long* tau_at;    // 2 x R entries
    CycleRecDev* log;
    long long log_cap;
    long long timeout_ns;
    int stall_barrier;
};

// Serving: one request of the ring, in device memory.  The host copies it
// in (and waits for the copy) before it publishes it by advancing *tail
// (host-mapped); the device block that claims it runs the instance, and the
// last block of its gang writes the outputs and sets done[slot] (host-mapped,
// system scope).
struct ServeSlot {
    RunParams P;                   // device pointers into the server's arena; P.inst = slot index
    double c[8], s[4];             // rate constants and Schloegl factors (FIM / RER)
    double cprime[8 * 8];          // perturbed parameter vectors of the RER
    double T_burn;                 // as given (the FIM / RER window starts here)
    int n_cprime, L;
    const double* gradU_n;         // toggle: d log(production) / d Hill exponent tables (arena)
    const double* gradV_n;
    double* out_hist;              // [nbins] histogram normalised by T_s
    double* out_fim;               // [64] FIM over [T_burn, T_s]
    double* out_rer;               // [8] RER over [T_burn, T_s]
    RunCtl* out_ctl;               // the control block at the end (statistics)
};

struct ServeDev {
    const ServeSlot* slots;        // device ring of cap entries
    int* done;                     // host-mapped: done[slot] = 1 when the request's outputs are written
    int cap, pad;
    const unsigned long long* tail;  // host-mapped: requests published
    unsigned long long* head;      // device: requests claimed
    unsigned long long* finished;  // device: requests whose outputs are written
    const int* stop;               // host-mapped: leave when set
    BatchDev bd;                   // idle set and mailboxes (remaining: unused counter)
    unsigned long long* progress;
    long long idle_exit_ns;        // blocks leave after the server has been idle this long
};

// ---- launchers (parrep_kernels.cu) ----
// (form: Form; the run kernel's is taken from p.form)
int kernel_attrs_form(int form, int kind, int* max_blocks_per_sm, int smem_bytes, int threads);
cudaError_t launch_run(const RunParams& p, int grid, int threads, int smem_bytes, cudaStream_t st);
int batch_attrs_form(int form, int* max_blocks_per_sm, int smem_bytes, int threads);
// zeroes the instances' control blocks and histograms, then launches the batch kernel
cudaError_t launch_batch(int form, const RunParams* d_params, int n, const int* d_off, const int2* d_items,
                         BatchDev bd, int grid, int threads, int smem_bytes, cudaStream_t st);
cudaError_t launch_batch_gather(const RunParams* d_params, int n, RunCtl* out, cudaStream_t st);
int serve_attrs_form(int form, int* max_blocks_per_sm, int smem_bytes, int threads);
cudaError_t launch_serve(int form, const ServeDev& sd, int grid, int threads, int smem_bytes, cudaStream_t st);
cudaError_t launch_dephase(const RunParams& p, int xt0, int xt1, int W, unsigned cycle, long long np,
                           int* out_states, int grid, int threads, cudaStream_t st);
cudaError_t launch_hist_normalise(const unsigned long long* pre, const unsigned long long* post, int n, double scale,
                                  double* out_pre, double* out_post, double* out_norm, cudaStream_t st);
// One sample of the stationary UQ over independent runs (Sec. IV.B): a
// completed run's network view and its post-burn time sums.
struct UqSample {
    NetDev net;
    const double* c;                  // rate constants (l)
    const unsigned long long* hist;   // post-burn fixed-point time sums
    const double* gradU_n;            // toggle: d log lambda / d n tables
    const double* gradV_n;
};
// Device result of the UQ reduction (the fields of parrep_uq_result).
struct UqOut {
    double iaf, mean_f;
    double fim[64], half[64], bound[8];
};
// Y[k] (window integral of f), Z[k][64] (FIM time average) per sample, then
// the moments, the FIM mean and half widths, and the bounds.
cudaError_t launch_uq(const UqSample* samples, int n, int L, const double* f, double window, const double* dirs,
                      int n_dirs, double* Y, double* Z, UqOut* out, double* dir_bounds, cudaStream_t st);
cudaError_t launch_fim_rer(const NetDev& net, const double* c, const double* s, const unsigned long long* hist,
                           const double* gradU_n, const double* gradV_n, const double* cprime, int n_cprime,
                           double* fim_out, double* rer_out, cudaStream_t st);
cudaError_t launch_ssa(const NetDev& net, int prec, long long n_traj, int x0, int x1, unsigned long long q_Tend,
                       unsigned long long seed, unsigned long long* hist, unsigned long long* events,
                       int* status, cudaStream_t st);
cudaError_t launch_ssa_trace(const NetDev& net, int prec, long long n_traj, int x0, int x1,
                             unsigned long long q_Tend, unsigned long long seed, long long max_steps, int* J,
                             int2* xs, unsigned long long* q, long long* n_out, int2* xf, int* status,
                             cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, long long n, uint32_t* out, cudaStream_t st);

}  // namespace parrep
