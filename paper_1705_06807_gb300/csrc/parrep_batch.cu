// Host side of the batch entry points (include/parrep.h): many ParRep
// instances in one persistent cooperative launch.  The scheduler sizes a gang
// of blocks for every instance, places the gangs longest-first on the
// co-resident grid and hands each block its ordered list of (instance, block
// index); the autotuner times candidate block shapes on a shortened copy of
// the batch; the launch sequence is captured once in a CUDA graph and
// replayed.  Every instance is an ordinary handle and ends the run holding
// the same results as parrep_run would have given it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "parrep.h"
#include "parrep_handle.h"
#include "parrep_internal.h"

using namespace parrep;

namespace {
thread_local std::string g_batch_create_error;
}

struct parrep_batch_s {
    std::vector<parrep_t> inst;
    parrep_batch_options opt{};
    int prec = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    // current block shape and its co-resident grid
    int threads = 0, RB = 0, grid = 0, smem = 0;
    int form = 0;  // kernel Form of the current shape
    bool tuned = false;
    std::vector<Plan> plans;
    std::vector<int> gang;
    // measured costs of every instance, pooled over the batch's runs:
    // simulated time, cycles, dephasing block-cycles and the other block-cycles
    std::vector<double> m_T, m_cycles, m_deph, m_rest;
    bool have_cost = false;
    // device buffers
    RunParams* d_params = nullptr;
    int* d_off = nullptr;
    int2* d_items = nullptr;
    RunCtl* d_ctl_out = nullptr;
    unsigned long long* d_progress = nullptr;
    int* d_remaining = nullptr;
    unsigned* d_idle = nullptr;
    int4* d_mail = nullptr;
    int off_cap = 0, items_cap = 0;
    // pinned host mirrors (the graph's copy nodes read and write these)
    RunParams* h_params = nullptr;
    int* h_off = nullptr;
    int2* h_items = nullptr;
    RunCtl* h_ctl_out = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // captured launch sequence and the shape it was captured for
    cudaGraphExec_t exec = nullptr;
    int g_threads = 0, g_grid = 0, g_smem = 0, g_items_cap = 0, g_off_cap = 0, g_form = -1;
    std::vector<int32_t> status;
    parrep_batch_info info{};
    std::string err;
};

static int bfail(parrep_batch_t b, int code, const std::string& msg) {
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return code;
}

static int bcuda(parrep_batch_t b, cudaError_t e, const char* what) {
    return bfail(b, PARREP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call)                                        \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);  \
    } while (0)

extern "C" void parrep_batch_default_options(parrep_batch_options* o) {
    memset(o, 0, sizeof(*o));
    o->block_threads = 0;
    o->replicas_per_block = 0;
    o->autotune = 1;
    o->use_graph = 1;
    o->tune_fraction = 0.05;
    o->wait_timeout_s = 10.0;
    o->stream = nullptr;
}

// ---------------------------------------------------------------------------
// work estimate and schedule
// ---------------------------------------------------------------------------

// Total propensity a0 at the instance's starting state in binary64 (the
// middle of the range when x_0 is drawn uniformly).
static double start_a0(parrep_t h) {
    const parrep_network& n = h->net;
    double x = n.x0_uniform_hi > 0 ? 0.5 * n.x0_uniform_hi : (double)n.x0[0];
    if (n.kind == PARREP_SCHLOGL) {
        const double a = x * (x - 1.0), c = a * (x - 2.0);
        return n.c[0] * n.s[0] * a + n.c[1] * n.s[1] * c + n.c[2] * n.s[2] + n.c[3] * n.s[3] * x;
    }
    const double U = x, V = n.x0_uniform_hi > 0 ? 0.5 * n.x0_uniform_hi : (double)n.x0[1];
    if (n.kind == PARREP_GENETIC) {
        // six channels at (xi, m, p) = (U mod 2, U / 2, V)
        const double xi = (double)((int)U & 1), m = (double)((int)U >> 1), p = V;
        const double hh = p * p / (p * p + n.c[7] * n.c[7]);
        const double F = n.c[3] + (n.c[4] - n.c[3]) * hh, G = n.c[6] - (n.c[6] - n.c[5]) * hh;
        return n.c[0] * xi + n.c[2] * m + n.c[2] * n.c[1] * m + p + F * (1.0 - xi) + G * xi;
    }
    return n.c[0] / (1.0 + pow(V, n.c[1])) + n.c[3] / (1.0 + pow(U, n.c[4])) + n.c[2] * U + n.c[5] * V;
}

// Estimated events of one run: holding times to T_end plus one dephasing
// stage of every replica (t_phase time units, or n_p jumps).
static double est_work(parrep_t h, double T_end) {
    const double a0 = std::max(start_a0(h), 1e-300);
    const double per_replica =
        h->opt.thresh_mode == PARREP_THRESH_STEPS ? h->t_phase : h->t_phase * a0;
    return T_end * a0 + (double)h->R * per_replica + 1.0;
}

// Adds the last run's block-cycles of every instance (the kernel's per-phase
// clocks summed over its blocks) to the pooled measurements.
static void record_costs(parrep_batch_t b, const double* T_end) {
    const int n = (int)b->inst.size();
    if (!b->have_cost) {
        b->m_T.assign(n, 0.0);
        b->m_cycles.assign(n, 0.0);
        b->m_deph.assign(n, 0.0);
        b->m_rest.assign(n, 0.0);
    }
    for (int i = 0; i < n; ++i) {
        const RunCtl& c = b->h_ctl_out[i];
        double tot = 0.0;
        for (int k = 0; k < 8; ++k) tot += (double)c.phase_cycles[k];  // 8..11 are parts of 0
        const double deph = (double)c.phase_cycles[1];
        b->m_T[i] += T_end[i];
        b->m_cycles[i] += (double)c.cycles;
        b->m_deph[i] += deph;
        b->m_rest[i] += tot - deph;
    }
    b->have_cost = true;
}

// Expected block-cycles of instance i to T_end, with room for the spread of
// its escape count: the other phases scale with T_end; every cycle adds one
// dephasing of all replicas, and the cycle count of a run is taken two
// standard deviations (Poisson) above its mean.
static double measured_work(parrep_batch_t b, int i, double T_end) {
    const double T = std::max(b->m_T[i], 1e-9);
    const double E = b->m_cycles[i] / T * T_end;
    const double per_cycle = b->m_cycles[i] > 0.0 ? b->m_deph[i] / b->m_cycles[i] : 0.0;
    return b->m_rest[i] / T * T_end + per_cycle * (E + 2.0 * sqrt(E) + 1.0);
}

// Gang sizes and the ordered (instance, local block) lists of every block.
// Work: the last run's measured cost, else an estimate.  An instance whose
// work exceeds the ideal makespan (total work / blocks) gets enough blocks to
// fit in it, up to one block per group of replicas.
static void make_schedule(parrep_batch_t b, const double* T_end) {
    const int n = (int)b->inst.size(), G = b->grid;
    std::vector<double> w(n), dur(n);
    double W = 0.0;
    for (int i = 0; i < n; ++i) {
        w[i] = b->have_cost ? std::max(measured_work(b, i, T_end[i]), 1.0) : est_work(b->inst[i], T_end[i]);
        W += w[i];
    }
    const double M = W / (double)G;
    b->gang.assign(n, 1);
    for (int i = 0; i < n; ++i) {
        const long long nvb = (b->inst[i]->R + b->plans[i].RB - 1) / b->plans[i].RB;
        long long g = (long long)ceil(w[i] / M - 1e-9);
        g = std::max(1LL, std::min(g, std::min(nvb, (long long)G)));
        b->gang[i] = (int)g;
        dur[i] = w[i] / (double)g;
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return dur[a] > dur[c]; });
    // longest first: each instance takes the g blocks that free up first
    std::vector<double> free_at(G, 0.0);
    std::vector<std::vector<int2>> lists(G);
    std::vector<int> blk(G);
    for (int i : order) {
        const int g = b->gang[i];
        std::iota(blk.begin(), blk.end(), 0);
        std::partial_sort(blk.begin(), blk.begin() + g, blk.end(),
                          [&](int x, int y) { return free_at[x] < free_at[y] || (free_at[x] == free_at[y] && x < y); });
        double start = 0.0;
        for (int k = 0; k < g; ++k) start = std::max(start, free_at[blk[k]]);
        for (int k = 0; k < g; ++k) {
            free_at[blk[k]] = start + dur[i];
            lists[blk[k]].push_back(make_int2(i, k));
        }
    }
    // every list is in assignment order, which is the order of start times on
    // that block, and one global order: no gang waits on a later one
    int m = 0;
    for (int k = 0; k < G; ++k) {
        b->h_off[k] = m;
        for (const int2& it : lists[k]) b->h_items[m++] = it;
    }
    b->h_off[G] = m;
    b->info.n_items = m;
    double mk = 0.0;
    for (int k = 0; k < G; ++k) mk = std::max(mk, free_at[k]);
    b->info.est_makespan = mk;
    b->info.est_balance = mk > 0.0 ? W / ((double)G * mk) : 1.0;
}

// ---------------------------------------------------------------------------
// block shape
// ---------------------------------------------------------------------------

// Per-instance layouts for blocks of `threads` with RB owners, the largest
// dynamic shared memory they need, and the co-resident grid.
static int set_shape(parrep_batch_t b, int threads, int RB, int form) {
    int dev = 0, nsm = 0;
    BCK(b, cudaGetDevice(&dev));
    BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int n = (int)b->inst.size();
    b->plans.assign(n, Plan{});
    int smem = 0;
    for (int i = 0; i < n; ++i) {
        parrep_t h = b->inst[i];
        Plan& pl = b->plans[i];
        memset(&pl, 0, sizeof(pl));
        // the mixed form runs each instance in its own layout (direct for the
        // genetic switch and from kDirectAutoReplicas replicas on)
        const int f = form != kFormF32Mixed ? form
                      : (h->R >= kDirectAutoReplicas || h->net.kind == PARREP_GENETIC) ? kFormF32Direct
                                                                                        : kFormF32Staged;
        pl.form = f;
        if (f == kFormF32Staged) {
            const int pipe = threads - RB >= 64 && !h->opt.serial_stages;
            int sz = -1;
            for (int with_hist = 1; with_hist >= 0 && sz < 0; --with_hist) {
                const int s = fast_layout(h, RB, threads, with_hist, pipe, pl);
                if (s <= 200 * 1024) sz = s;
            }
            if (sz < 0) return bfail(b, PARREP_ENOMEM, "an instance's tables do not fit in shared memory");
            pl.threads = threads;
            pl.smem = sz;
            const int S = h->opt.chunk_steps > 0 ? h->opt.chunk_steps : default_chunk(true, h->R);
            pl.S = ((S + pl.B - 1) / pl.B) * pl.B;
        } else {
            pl.threads = threads;
            pl.RB = threads;
            pl.B = 0;
            pl.S = h->opt.chunk_steps > 0 ? h->opt.chunk_steps : default_chunk(false, h->R);
            pl.off_tab = pl.off_buf = pl.off_trace = pl.off_live = pl.off_nvalid = -1;
            pl.off_limbs = pl.off_inv = pl.off_rng = pl.off_decp = pl.off_thr = -1;
            pl.use_smem_hist = h->nbins * 8 <= (form == kFormF32Direct ? kDirectSmemHistLimit : kSmemHistLimit);
            pl.form = f;
            pl.smem = pl.use_smem_hist ? h->nbins * 8 : 0;
        }
        if (pl.S > kMaxChunk) return bfail(b, PARREP_EINVAL, "chunk_steps too large");
        smem = std::max(smem, pl.smem);
    }
    int per_sm = 0;
    const int ea = batch_attrs_form(form, &per_sm, smem, threads);
    if (ea != 0) return bcuda(b, (cudaError_t)ea, "batch kernel attributes");
    if (per_sm < 1) return bfail(b, PARREP_ENOMEM, "the batch kernel does not fit on one SM");
    b->threads = threads;
    b->RB = RB;
    b->form = form;
    b->smem = smem;
    b->grid = per_sm * nsm;
    b->info.block_threads = threads;
    b->info.replicas_per_block = RB;
    b->info.grid_blocks = b->grid;
    b->info.f32_layout = form == kFormF32Staged  ? PARREP_F32_STAGED
                         : form == kFormF32Direct ? PARREP_F32_DIRECT
                         : form == kFormF32Mixed  ? PARREP_F32_MIXED
                                                  : 0;
    // buffers sized for this grid
    const int items_cap = n * b->grid, off_cap = b->grid + 1;
    if (items_cap > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        if (b->h_items) cudaFreeHost(b->h_items);
        b->d_items = nullptr;
        b->h_items = nullptr;
        BCK(b, cudaMalloc((void**)&b->d_items, sizeof(int2) * items_cap));
        BCK(b, cudaMallocHost((void**)&b->h_items, sizeof(int2) * items_cap));
        b->items_cap = items_cap;
    }
    if (off_cap > b->off_cap) {
        if (b->d_off) cudaFree(b->d_off);
        if (b->h_off) cudaFreeHost(b->h_off);
        if (b->d_idle) cudaFree(b->d_idle);
        if (b->d_mail) cudaFree(b->d_mail);
        b->d_off = nullptr;
        b->h_off = nullptr;
        b->d_idle = nullptr;
        b->d_mail = nullptr;
        BCK(b, cudaMalloc((void**)&b->d_off, sizeof(int) * off_cap));
        BCK(b, cudaMallocHost((void**)&b->h_off, sizeof(int) * off_cap));
        BCK(b, cudaMalloc((void**)&b->d_idle, sizeof(unsigned) * ((off_cap + 31) / 32)));
        BCK(b, cudaMalloc((void**)&b->d_mail, sizeof(int4) * off_cap));
        b->off_cap = off_cap;
    }
    return PARREP_OK;
}

// ---------------------------------------------------------------------------
// one run
// ---------------------------------------------------------------------------

// The launch sequence on b->st (also what the graph captures).
static int enqueue(parrep_batch_t b) {
    const int n = (int)b->inst.size();
    BCK(b, cudaMemcpyAsync(b->d_params, b->h_params, sizeof(RunParams) * n, cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaMemcpyAsync(b->d_off, b->h_off, sizeof(int) * b->off_cap, cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaMemcpyAsync(b->d_items, b->h_items, sizeof(int2) * b->items_cap, cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaMemsetAsync(b->d_progress, 0, sizeof(unsigned long long), b->st));
    BatchDev bd{b->d_remaining, b->d_idle, b->d_mail, nullptr, nullptr, 0, 0};
    BCK(b, launch_batch(b->form, b->d_params, n, b->d_off, b->d_items, bd, b->grid, b->threads, b->smem, b->st));
    BCK(b, launch_batch_gather(b->d_params, n, b->d_ctl_out, b->st));
    BCK(b, cudaMemcpyAsync(b->h_ctl_out, b->d_ctl_out, sizeof(RunCtl) * n, cudaMemcpyDeviceToHost, b->st));
    return PARREP_OK;
}

static int run_once(parrep_batch_t b, const double* T_end, const uint64_t* seed, bool graph, float* ms_out) {
    const int n = (int)b->inst.size();
    make_schedule(b, T_end);
    for (int i = 0; i < n; ++i) {
        parrep_t h = b->inst[i];
        Plan pl = b->plans[i];
        pl.grid = b->gang[i];
        RunParams p;
        int rc = run_params(h, T_end[i], seed[i], pl, p);
        if (rc != PARREP_OK) return bfail(b, rc, std::string("instance ") + std::to_string(i) + ": " + h->err);
        p.progress = b->d_progress;
        p.timeout_ns = (long long)(b->opt.wait_timeout_s * 1e9);
        p.batch = BatchDev{b->d_remaining, b->d_idle, b->d_mail, nullptr, nullptr, 0, 0};
        p.inst = i;
        b->h_params[i] = p;
    }
    if (graph) {
        const bool same = b->exec && b->g_threads == b->threads && b->g_grid == b->grid && b->g_smem == b->smem &&
                          b->g_items_cap == b->items_cap && b->g_off_cap == b->off_cap && b->g_form == b->form;
        if (!same) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            BCK(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue(b);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->st, &g);
            if (rc != PARREP_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ec != cudaSuccess) return bcuda(b, ec, "cudaStreamEndCapture");
            const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                b->exec = nullptr;
                return bcuda(b, ei, "cudaGraphInstantiate");
            }
            b->g_threads = b->threads;
            b->g_grid = b->grid;
            b->g_smem = b->smem;
            b->g_items_cap = b->items_cap;
            b->g_off_cap = b->off_cap;
            b->g_form = b->form;
        }
        BCK(b, cudaEventRecord(b->ev0, b->st));
        BCK(b, cudaGraphLaunch(b->exec, b->st));
        BCK(b, cudaEventRecord(b->ev1, b->st));
    } else {
        BCK(b, cudaEventRecord(b->ev0, b->st));
        const int rc = enqueue(b);
        if (rc != PARREP_OK) return rc;
        BCK(b, cudaEventRecord(b->ev1, b->st));
    }
    BCK(b, cudaStreamSynchronize(b->st));
    float ms = 0.f;
    BCK(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    *ms_out = ms;
    b->info.graph = graph ? 1 : 0;
    return PARREP_OK;
}

// Candidate shapes: {threads, RB, form}.  FP32 staged: RB owners + helpers;
// FP32 direct and FP64: one replica a thread (RB = threads); FP32 mixed: each
// instance staged with RB owners or direct with all threads as owners.  The
// FP32 auto layout is the mixed one: it runs a batch without large or genetic
// instances exactly as the staged layout does.
struct Shape {
    int threads, RB, form;
};

static std::vector<Shape> candidates(parrep_batch_t b) {
    std::vector<Shape> c;
    const int T = b->opt.block_threads, RB = b->opt.replicas_per_block;
    if (b->prec == PARREP_FP32) {
        const int lay = b->opt.f32_layout;
        if (lay == PARREP_F32_STAGED || lay == PARREP_F32_AUTO || lay == PARREP_F32_MIXED) {
            const int form = lay == PARREP_F32_STAGED ? kFormF32Staged : kFormF32Mixed;
            const int all[][2] = {{384, 64}, {384, 32}, {384, 128}, {256, 32}, {256, 64}};
            for (auto& s : all)
                if ((T == 0 || s[0] == T) && (RB == 0 || s[1] == RB)) c.push_back({s[0], s[1], form});
            if (c.empty() && (T == 0 || RB == 0 || RB < T)) c.push_back({T ? T : 384, RB ? RB : 64, form});
        } else {
            const int all[] = {kDirectThreads, 128};
            for (int t : all)
                if ((T == 0 || t == T) && (RB == 0 || RB == t)) c.push_back({t, t, kFormF32Direct});
            if (c.empty()) c.push_back({kDirectThreads, kDirectThreads, kFormF32Direct});
        }
    } else {
        const int all[] = {128, 256, 64};
        for (int t : all)
            if (T == 0 || t == T) c.push_back({t, t, kFormF64});
        if (c.empty()) c.push_back({T, T, kFormF64});
    }
    if (!b->opt.autotune) c.resize(1);
    return c;
}

static int autotune(parrep_batch_t b, const double* T_end, const uint64_t* seed) {
    const auto cand = candidates(b);
    const int n = (int)b->inst.size();
    auto t0 = std::chrono::steady_clock::now();
    if (cand.size() > 1) {
        std::vector<double> Tt(n), burn(n);
        for (int i = 0; i < n; ++i) {
            Tt[i] = T_end[i] * b->opt.tune_fraction;
            burn[i] = b->inst[i]->opt.T_burn;
            b->inst[i]->opt.T_burn = burn[i] * b->opt.tune_fraction;
        }
        float best = 0.f;
        int best_k = -1, rc = PARREP_OK;
        if (!b->have_cost) {
            // one unscored run to measure the instances' costs, so that every
            // candidate is timed with a measured schedule
            rc = set_shape(b, cand[0].threads, cand[0].RB, cand[0].form);
            float ms = 0.f;
            if (rc == PARREP_OK) rc = run_once(b, Tt.data(), seed, false, &ms);
            if (rc == PARREP_OK) record_costs(b, Tt.data());
            if (rc == PARREP_ENOMEM) rc = PARREP_OK;
        }
        for (size_t k = 0; k < cand.size() && rc == PARREP_OK; ++k) {
            rc = set_shape(b, cand[k].threads, cand[k].RB, cand[k].form);
            if (rc == PARREP_ENOMEM) {  // this shape does not fit some instance: skip it
                rc = PARREP_OK;
                continue;
            }
            if (rc != PARREP_OK) break;
            float ms = 0.f;
            rc = run_once(b, Tt.data(), seed, false, &ms);
            if (rc != PARREP_OK) break;
            record_costs(b, Tt.data());
            b->info.tuned_trials += 1;
            if (best_k < 0 || ms < best) {
                best = ms;
                best_k = (int)k;
            }
        }
        for (int i = 0; i < n; ++i) b->inst[i]->opt.T_burn = burn[i];
        if (rc != PARREP_OK) return rc;
        if (best_k < 0) return bfail(b, PARREP_ENOMEM, "no candidate block shape fits every instance");
        int rc2 = set_shape(b, cand[best_k].threads, cand[best_k].RB, cand[best_k].form);
        if (rc2 != PARREP_OK) return rc2;
    } else {
        int rc = set_shape(b, cand[0].threads, cand[0].RB, cand[0].form);
        if (rc != PARREP_OK) return rc;
    }
    b->tuned = true;
    b->info.tune_ms =
        (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PARREP_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------

static void batch_free(parrep_batch_t b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    void* dev[] = {b->d_params, b->d_off, b->d_items, b->d_ctl_out, b->d_progress, b->d_remaining, b->d_idle,
                   b->d_mail};
    for (void* p : dev)
        if (p) cudaFree(p);
    void* host[] = {b->h_params, b->h_off, b->h_items, b->h_ctl_out};
    for (void* p : host)
        if (p) cudaFreeHost(p);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
}

extern "C" int parrep_batch_create(const parrep_t* instances, int32_t n, const parrep_batch_options* opt,
                                   parrep_batch_t* out) {
    if (!out) return bfail(nullptr, PARREP_EINVAL, "out is null");
    *out = nullptr;
    if (!instances || n < 1) return bfail(nullptr, PARREP_EINVAL, "need n >= 1 instances");
    parrep_batch_options o;
    parrep_batch_default_options(&o);
    if (opt) o = *opt;
    if (o.block_threads < 0 || o.block_threads > kMaxThreads || o.block_threads % 32 != 0)
        return bfail(nullptr, PARREP_EINVAL, "block_threads must be a multiple of 32 up to 384 (0 = autotune)");
    if (o.f32_layout < PARREP_F32_AUTO || o.f32_layout > PARREP_F32_MIXED)
        return bfail(nullptr, PARREP_EINVAL, "f32_layout");
    const int rb = o.replicas_per_block;
    if (!(rb == 0 || rb == 32 || rb == 64 || rb == 128 || rb == 256))
        return bfail(nullptr, PARREP_EINVAL, "replicas_per_block must be 0, 32, 64, 128 or 256");
    if (!(o.tune_fraction > 0.0 && o.tune_fraction <= 1.0)) return bfail(nullptr, PARREP_EINVAL, "tune_fraction");
    if (!(o.wait_timeout_s > 0.0) || !(o.wait_timeout_s <= 3600.0))
        return bfail(nullptr, PARREP_EINVAL, "wait_timeout_s");
    std::vector<parrep_t> v(instances, instances + n);
    for (int i = 0; i < n; ++i) {
        if (!v[i]) return bfail(nullptr, PARREP_EINVAL, "null instance handle");

        if (v[i]->opt.precision != v[0]->opt.precision)
            return bfail(nullptr, PARREP_EINVAL, "instances of one batch need the same precision");
        if (v[i]->opt.precision == PARREP_FP32 && v[i]->net.kind == PARREP_GENETIC &&
            o.f32_layout == PARREP_F32_STAGED)
            return bfail(nullptr, PARREP_EINVAL,
                         "the genetic switch's FP32 form needs the direct, mixed or auto layout (f32_layout)");
    }
    std::vector<parrep_t> sorted(v);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return bfail(nullptr, PARREP_EINVAL, "an instance appears twice");
    if (v[0]->opt.precision == PARREP_FP32 && o.block_threads > 0 && rb > 0 && o.block_threads < rb)
        return bfail(nullptr, PARREP_EINVAL, "block_threads < replicas_per_block");
    parrep_batch_s* b = new parrep_batch_s();
    b->inst = v;
    b->opt = o;
    b->prec = v[0]->opt.precision;
    b->status.assign(n, 0);
    cudaError_t e = cudaSuccess;
    if (o.stream) {
        b->st = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_params, sizeof(RunParams) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ctl_out, sizeof(RunCtl) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_progress, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_remaining, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_params, sizeof(RunParams) * n);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctl_out, sizeof(RunCtl) * n);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e != cudaSuccess) {
        std::string m = std::string("parrep_batch_create: ") + cudaGetErrorString(e);
        batch_free(b);
        delete b;
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? PARREP_ENOMEM : PARREP_ECUDA, m);
    }
    *out = b;
    return PARREP_OK;
}

extern "C" int parrep_batch_run(parrep_batch_t b, const double* T_end, const uint64_t* seed) {
    if (!b || !T_end || !seed) return PARREP_EINVAL;
    const int n = (int)b->inst.size();
    for (int i = 0; i < n; ++i) {
        parrep_t h = b->inst[i];
        if (h->opt.precision != b->prec)
            return bfail(b, PARREP_EINVAL, "an instance's precision changed after parrep_batch_create");
        const int rc = run_checks(h, T_end[i]);
        if (rc != PARREP_OK) return bfail(b, rc, std::string("instance ") + std::to_string(i) + ": " + h->err);
    }
    if (!b->tuned) {
        const int rc = autotune(b, T_end, seed);
        if (rc != PARREP_OK) return rc;
    }
    float ms = 0.f;
    int rc = run_once(b, T_end, seed, b->opt.use_graph != 0, &ms);
    if (rc != PARREP_OK) return rc;
    b->info.kernel_ms = ms;
    record_costs(b, T_end);
    int first = PARREP_OK;
    for (int i = 0; i < n; ++i) {
        Plan pl = b->plans[i];
        pl.grid = b->gang[i];
        RunCtl c = b->h_ctl_out[i];
        if (c.status == 0 && !c.done) c.status = PARREP_ETIMEOUT;  // the instance never finished
        b->status[i] = run_finish(b->inst[i], c, T_end[i], pl, ms);
        if (b->status[i] != PARREP_OK && first == PARREP_OK) {
            first = b->status[i];
            b->err = std::string("instance ") + std::to_string(i) + ": " + b->inst[i]->err;
        }
    }
    return first;
}

extern "C" int parrep_batch_status(parrep_batch_t b, int32_t* status_out) {
    if (!b || !status_out) return PARREP_EINVAL;
    for (size_t i = 0; i < b->status.size(); ++i) status_out[i] = b->status[i];
    return PARREP_OK;
}

extern "C" int parrep_batch_info_get(parrep_batch_t b, parrep_batch_info* out) {
    if (!b || !out) return PARREP_EINVAL;
    *out = b->info;
    return PARREP_OK;
}

extern "C" void parrep_batch_destroy(parrep_batch_t b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    batch_free(b);
    delete b;
}

extern "C" const char* parrep_batch_last_error(parrep_batch_t b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}
