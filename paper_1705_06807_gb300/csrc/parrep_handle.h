// Host-side internals shared by the single-run (parrep_api.cu) and the batch
// (parrep_batch.cu) halves of the C ABI.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "parrep.h"
#include "parrep_internal.h"

namespace parrep {

constexpr long long kLogCap = 1 << 16;
constexpr int kMaxChunk = 1 << 16;
constexpr int kSmemHistLimit = 160 * 1024;
// the binary32 direct layout keeps three blocks per SM: a block's histogram
// stays in shared memory only up to this size, larger ones go to global memory
constexpr int kDirectSmemHistLimit = 64 * 1024;
// Longest chunk of the FP32 form between escape votes (chunks start at one
// sub-chunk in each cycle and double): fewer grid barriers per run against
// more discarded work after an escape; 2048 measured best of 512..2048 on the
// n = 4096 Schloegl run.
constexpr int kDefaultChunkF32 = 2048;
// Default chunk length: kDefaultChunkF32 (staged) or 256 (one thread per
// replica), halved down to 128 while a chunk would hold more than 2^23
// replica-steps -- an escape discards about half a chunk of every replica's
// steps, so instances with many replicas vote more often.  Where chunks end
// does not change any result.
inline int default_chunk(bool staged, long long R) {
    long long s = staged ? kDefaultChunkF32 : 256;
    while (s > 128 && s * R > (1LL << 23)) s >>= 1;
    return (int)s;
}

}  // namespace parrep

struct parrep_s {
    parrep_network net;
    parrep_regions reg;
    int64_t R = 0;
    double t_corr = 0, t_phase = 0;
    parrep_options opt;
    int nbins = 0, L = 4;
    parrep::NetDev nd{};
    // device buffers
    double *d_prodU_d = nullptr, *d_prodV_d = nullptr;
    float *d_prodU_f = nullptr, *d_prodV_f = nullptr;
    double *d_gradU_n = nullptr, *d_gradV_n = nullptr, *d_c = nullptr, *d_s = nullptr;
    parrep::RunCtl* d_ctl = nullptr;
    unsigned long long *d_hist_pre = nullptr, *d_hist_post = nullptr, *d_step_sum = nullptr, *d_tau_at = nullptr;
    int2* d_xstate = nullptr;  // [3 R]: replica state, chunk-start state, exit state
    parrep::CycleRecDev* d_log = nullptr;
    double *d_out = nullptr, *d_out2 = nullptr, *d_fim = nullptr, *d_rer = nullptr, *d_cprime = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // last run
    bool has_run = false;
    parrep::RunCtl h_ctl{};
    double T_end = 0, T_burn = 0;
    parrep_stats stats{};
    std::string err;
};

namespace parrep {

// Launch plan of parrep_run.  FP64 form: one replica per thread.  FP32 form:
// blocks of T threads of which the first RB own replicas (RB a power of two,
// >= 32), the smallest RB whose grid is co-resident; B staged steps (staged_sub_chunk).
struct Plan {
    int form;  // Form (parrep_internal.h)
    int threads, grid, smem, RB, log2RB, B, S, use_smem_hist;
    int off_tab, off_buf, off_trace, off_live, off_nvalid;
    int off_limbs, off_inv, off_rng, off_decp;
    int off_thr;
    int pipelined;
};

int fail(parrep_t h, int code, const std::string& msg);
// network and region checks of parrep_create (1 = valid, else why is set)
int check_network(const parrep_network* net, const parrep_regions* reg, std::string& why);
// the kernels' view of a network and the host-built toggle tables
void build_net(const parrep_network* net, const parrep_regions* reg, NetDev& nd, std::vector<double>& pU,
               std::vector<double>& pV, std::vector<double>& gU, std::vector<double>& gV);
int cuda_fail(parrep_t h, cudaError_t e, const char* what);
int align16(int x);
// shared-memory layout of the FP32 form for RB owners in blocks of `threads`
int fast_layout(parrep_t h, int RB, int threads, int with_hist, int pipelined, Plan& pl);
int run_checks(parrep_t h, double T_end);
// kernel Form of the handle's runs (binary64, binary32 staged or direct)
int f32_form(parrep_t h);
// the FP32 form's auto layout is direct from this many replicas on
constexpr long long kDirectAutoReplicas = 16384;
int run_params(parrep_t h, double T_end, uint64_t seed, const Plan& pl, RunParams& p);
int run_finish(parrep_t h, const RunCtl& c, double T_end, const Plan& pl, float ms);
// the statistics a control block holds (launch shape and timing left zero)
void stats_from_ctl(const RunCtl& c, parrep_stats& s);

}  // namespace parrep
