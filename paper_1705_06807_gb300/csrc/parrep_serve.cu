// Host side of the serving entry points (include/parrep.h): a request loop
// with continuous batching.  Requests are queued by client threads; a host
// thread admits them in arrival order while ring slots and arena memory
// allow (first fit), copies each into the device ring and publishes it;
// the persistent serve kernel (parrep_kernels.cu) picks published requests
// up on idle blocks, grows their gangs at cycle starts and flags them done.
// The host thread relaunches the kernel when it has left while requests
// wait, and records completions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "parrep.h"
#include "parrep_handle.h"
#include "parrep_internal.h"

using namespace parrep;

namespace {

thread_local std::string g_server_create_error;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) of the device arena.
class Arena {
public:
    void init(size_t size) {
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    parrep_request r{};
    std::vector<double> cprime;
    int state = PARREP_REQ_QUEUED;
    int slot = -1;
    size_t off = 0, bytes = 0;
    int nbins = 0, L = 4;
    double t_submit = 0, t_done = 0;
    // device outputs in the arena
    double *d_hist = nullptr, *d_fim = nullptr, *d_rer = nullptr;
    RunCtl* d_ctl_out = nullptr;
};

}  // namespace

struct parrep_server_s {
    parrep_server_options opt{};
    int threads = 0, RB = 0, smem = 0, grid = 0;
    int form = 0;  // kernel Form of the serve kernel
    char* d_arena = nullptr;
    Arena arena;
    // ring of requests in device memory, a host staging copy of one slot, and
    // the host-mapped flags (host pointers; the device uses the same addresses)
    ServeSlot* d_slots = nullptr;
    ServeSlot* h_slot = nullptr;
    int* done = nullptr;
    unsigned long long* tail = nullptr;
    int* stop = nullptr;
    // device state of the serve kernel
    unsigned long long* d_head = nullptr;
    unsigned long long* d_finished = nullptr;
    unsigned* d_idle = nullptr;
    int4* d_mail = nullptr;
    int* d_unused = nullptr;
    unsigned long long* d_progress = nullptr;
    cudaStream_t st = nullptr, cp = nullptr;
    cudaEvent_t ev_end = nullptr;
    bool kernel_live = false;
    // bookkeeping
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool quit = false;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<int64_t> queue;
    std::vector<int64_t> slot_owner;
    int64_t next_id = 1;
    unsigned long long published = 0;
    parrep_server_stats stats{};
    std::string err;
    int dev = 0;
};

static int sfail(parrep_server_t s, int code, const std::string& msg) {
    if (s) s->err = msg;
    else g_server_create_error = msg;
    return code;
}

extern "C" void parrep_server_default_options(parrep_server_options* o) {
    memset(o, 0, sizeof(*o));
    o->precision = PARREP_FP32;
    o->block_threads = 0;
    o->replicas_per_block = 0;
    o->ring = 4096;
    o->f32_layout = PARREP_F32_MIXED;
    o->arena_bytes = 4ll << 30;
    o->log_cap = 4096;
    o->idle_exit_s = 0.05;
    o->wait_timeout_s = 10.0;
}

// Arena bytes of a request: control block and its end copy, histograms and
// outputs, step sums, replica state, cycle log, toggle tables.
static size_t request_bytes(const parrep_request& r, int64_t log_cap) {
    const size_t nb = (size_t)(r.net.hist_max[0] + 1) * (size_t)(r.net.hist_max[1] + 1);
    const size_t R = (size_t)r.n_replicas;
    size_t b = 0;
    b += align256(sizeof(RunCtl)) * 2;
    b += align256(nb * 8) * 3;
    b += align256(64 * 8) + align256(8 * 8);
    b += align256(sizeof(unsigned long long) * kMaxChunk);
    b += align256(sizeof(unsigned long long) * 2 * R);
    b += align256(sizeof(int2) * 3 * R);
    b += align256(sizeof(CycleRecDev) * (size_t)log_cap);
    if (r.net.kind == PARREP_TOGGLE) {
        const size_t nu = (size_t)r.net.hist_max[1] + 1, nv = (size_t)r.net.hist_max[0] + 1;
        b += 2 * (align256(nu * 8) + align256(nv * 8)) + align256(nu * 4) + align256(nv * 4);
    } else if (r.net.kind == PARREP_GENETIC) {
        const size_t np = (size_t)r.net.hist_max[1] + 1;
        b += 2 * align256(np * 8) + 2 * align256(np * 4);  // F(p), G(p) in binary64 and binary32
    }
    return b;
}

// Builds the request's instance in its arena block and fills its ring slot.
// Called by the host thread with the lock held.
static int admit(parrep_server_t s, Request& q, int slot) {
    const parrep_request& r = q.r;
    parrep_s h;
    h.net = r.net;
    h.reg = r.regions;
    h.R = r.n_replicas;
    h.t_corr = r.t_corr;
    h.t_phase = r.t_phase;
    parrep_default_options(&h.opt);
    h.opt.precision = s->opt.precision;
    h.opt.thresh_mode = r.thresh_mode;
    h.opt.fv_group = r.fv_group > 0 ? r.fv_group : 32;
    h.opt.chunk_steps = r.chunk_steps;
    h.opt.T_burn = r.T_burn;
    h.nbins = q.nbins;
    h.L = q.L;
    std::vector<double> pU, pV, gU, gV;
    build_net(&r.net, &r.regions, h.nd, pU, pV, gU, gV);
    char* base = s->d_arena + q.off;
    size_t o = 0;
    auto take = [&](size_t n) {
        char* p = base + o;
        o += align256(n);
        return p;
    };
    const size_t nb = (size_t)q.nbins, R = (size_t)r.n_replicas;
    h.d_ctl = (RunCtl*)take(sizeof(RunCtl));
    q.d_ctl_out = (RunCtl*)take(sizeof(RunCtl));
    h.d_hist_pre = (unsigned long long*)take(nb * 8);
    h.d_hist_post = (unsigned long long*)take(nb * 8);
    q.d_hist = (double*)take(nb * 8);
    q.d_fim = (double*)take(64 * 8);
    q.d_rer = (double*)take(8 * 8);
    h.d_step_sum = (unsigned long long*)take(sizeof(unsigned long long) * kMaxChunk);
    h.d_tau_at = (unsigned long long*)take(sizeof(unsigned long long) * 2 * R);
    h.d_xstate = (int2*)take(sizeof(int2) * 3 * R);
    h.d_log = (CycleRecDev*)take(sizeof(CycleRecDev) * (size_t)s->opt.log_cap);
    const double* d_gU = nullptr;
    const double* d_gV = nullptr;
    cudaError_t e = cudaSuccess;
    if (r.net.kind == PARREP_TOGGLE) {
        const size_t nu = pU.size(), nv = pV.size();
        double* pUd = (double*)take(nu * 8);
        double* pVd = (double*)take(nv * 8);
        double* gUd = (double*)take(nu * 8);
        double* gVd = (double*)take(nv * 8);
        float* pUf = (float*)take(nu * 4);
        float* pVf = (float*)take(nv * 4);
        std::vector<float> fU(nu), fV(nv);
        for (size_t i = 0; i < nu; ++i) fU[i] = (float)pU[i];
        for (size_t i = 0; i < nv; ++i) fV[i] = (float)pV[i];
        e = cudaMemcpyAsync(pUd, pU.data(), nu * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pVd, pV.data(), nv * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gUd, gU.data(), nu * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gVd, gV.data(), nv * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pUf, fU.data(), nu * 4, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pVf, fV.data(), nv * 4, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->cp);
        h.nd.prodU_d = pUd;
        h.nd.prodV_d = pVd;
        h.nd.prodU_f = pUf;
        h.nd.prodV_f = pVf;
        d_gU = gUd;
        d_gV = gVd;
    } else if (r.net.kind == PARREP_GENETIC) {
        // the switching rates F(p), G(p) as tables over p, in binary64 (the
        // binary64 form and the FIM / RER) and binary32 (the binary32 form)
        const size_t np = pU.size();
        double* Fd = (double*)take(np * 8);
        double* Gd = (double*)take(np * 8);
        float* Ff = (float*)take(np * 4);
        float* Gf = (float*)take(np * 4);
        std::vector<float> fF(np), fG(np);
        for (size_t i = 0; i < np; ++i) {
            fF[i] = (float)pU[i];
            fG[i] = (float)pV[i];
        }
        e = cudaMemcpyAsync(Fd, pU.data(), np * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Gd, pV.data(), np * 8, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Ff, fF.data(), np * 4, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Gf, fG.data(), np * 4, cudaMemcpyHostToDevice, s->cp);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->cp);
        h.nd.prodU_d = Fd;
        h.nd.prodV_d = Gd;
        h.nd.prodU_f = Ff;
        h.nd.prodV_f = Gf;
    }
    // (the serve kernel's claiming block clears the control block and the
    // histograms: a memset here would be a kernel that waits for free SMs)
    if (e != cudaSuccess) return sfail(s, PARREP_ECUDA, std::string("admission: ") + cudaGetErrorString(e));
    // launch shape of one gang member
    Plan pl;
    memset(&pl, 0, sizeof(pl));
    // the mixed form runs each request in its own layout (direct for the
    // genetic switch and from kDirectAutoReplicas replicas on)
    pl.form = s->form != kFormF32Mixed ? s->form
              : (r.n_replicas >= kDirectAutoReplicas || r.net.kind == PARREP_GENETIC) ? kFormF32Direct
                                                                                        : kFormF32Staged;
    if (pl.form == kFormF32Staged) {
        const int pipe = s->threads - s->RB >= 64;
        int sz = -1;
        for (int with_hist = 1; with_hist >= 0 && sz < 0; --with_hist) {
            const int z = fast_layout(&h, s->RB, s->threads, with_hist, pipe, pl);
            if (z <= s->smem) sz = z;
        }
        if (sz < 0) return sfail(s, PARREP_ENOMEM, "the request's tables do not fit the serve kernel's shared memory");
        pl.smem = sz;
        const int S = r.chunk_steps > 0 ? r.chunk_steps : default_chunk(true, r.n_replicas);
        pl.S = ((S + pl.B - 1) / pl.B) * pl.B;
    } else {
        pl.RB = s->threads;
        pl.S = r.chunk_steps > 0 ? r.chunk_steps : default_chunk(false, r.n_replicas);
        pl.off_tab = pl.off_buf = pl.off_trace = pl.off_live = pl.off_nvalid = -1;
        pl.off_limbs = pl.off_inv = pl.off_rng = pl.off_decp = pl.off_thr = -1;
        pl.use_smem_hist = (long long)nb * 8 <= (long long)s->smem;
        pl.smem = pl.use_smem_hist ? (int)nb * 8 : 0;
    }
    pl.threads = s->threads;
    pl.grid = 1;  // the claiming block; the gang grows at cycle starts
    RunParams p;
    const int rc = run_params(&h, r.T_end, r.seed, pl, p);
    if (rc != PARREP_OK) return sfail(s, rc, h.err);
    p.progress = s->d_progress;
    p.timeout_ns = (long long)(s->opt.wait_timeout_s * 1e9);
    p.batch = BatchDev{s->d_unused, s->d_idle, s->d_mail, s->tail, s->d_head, s->grid / 8, 0};
    p.inst = slot;
    p.log_cap = s->opt.log_cap;
    ServeSlot& sl = *s->h_slot;
    memset(&sl, 0, sizeof(sl));
    sl.P = p;
    for (int i = 0; i < 8; ++i) sl.c[i] = r.net.c[i];
    for (int i = 0; i < 4; ++i) sl.s[i] = r.net.s[i];
    memset(sl.cprime, 0, sizeof(sl.cprime));
    for (size_t i = 0; i < q.cprime.size() && i < 64; ++i) sl.cprime[i] = q.cprime[i];
    sl.T_burn = r.T_burn;
    sl.n_cprime = r.n_cprime;
    sl.L = q.L;
    sl.gradU_n = d_gU;
    sl.gradV_n = d_gV;
    sl.out_hist = q.d_hist;
    sl.out_fim = q.d_fim;
    sl.out_rer = q.d_rer;
    sl.out_ctl = q.d_ctl_out;
    ((volatile int*)s->done)[slot] = 0;
    e = cudaMemcpyAsync(s->d_slots + slot, &sl, sizeof(ServeSlot), cudaMemcpyHostToDevice, s->cp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cp);
    if (e != cudaSuccess) return sfail(s, PARREP_ECUDA, std::string("admission: ") + cudaGetErrorString(e));
    return PARREP_OK;
}

// One pass of the host thread (lock held): completions, admissions, launch.
static void serve_pass(parrep_server_t s) {
    for (auto& kv : s->reqs) {
        Request& q = *kv.second;
        if (q.state == PARREP_REQ_RUNNING && ((volatile int*)s->done)[q.slot]) {
            std::atomic_thread_fence(std::memory_order_acquire);
            q.state = PARREP_REQ_DONE;
            q.t_done = now_s();
            s->stats.completed += 1;
            s->stats.running -= 1;
        }
    }
    while (!s->queue.empty()) {
        Request& q = *s->reqs[s->queue.front()];
        const int slot = (int)(s->published % (unsigned long long)s->opt.ring);
        if (s->slot_owner[slot] >= 0) break;  // the ring holds unread results
        if (!s->arena.alloc(q.bytes, &q.off)) break;
        const int rc = admit(s, q, slot);
        if (rc != PARREP_OK) {
            // a request that fails admission is done, with no results
            s->arena.release(q.off, q.bytes);
            q.bytes = 0;
            q.state = PARREP_REQ_DONE;
            q.slot = -1;
            q.t_done = now_s();
            s->queue.pop_front();
            s->stats.queued -= 1;
            s->stats.completed += 1;
            continue;
        }
        q.slot = slot;
        s->slot_owner[slot] = s->queue.front();
        q.state = PARREP_REQ_RUNNING;
        s->queue.pop_front();
        s->stats.queued -= 1;
        s->stats.running += 1;
        s->stats.admitted += 1;
        std::atomic_thread_fence(std::memory_order_release);
        s->published += 1;
        ((volatile unsigned long long*)s->tail)[0] = s->published;
    }
    if (s->kernel_live && cudaEventQuery(s->ev_end) == cudaSuccess) s->kernel_live = false;
    if (!s->kernel_live && s->stats.running > 0) {
        // requests wait and no serve kernel is on the device: launch one
        ServeDev sd;
        sd.slots = s->d_slots;
        sd.done = s->done;
        sd.cap = s->opt.ring;
        sd.pad = 0;
        sd.tail = s->tail;
        sd.head = s->d_head;
        sd.finished = s->d_finished;
        sd.stop = s->stop;
        sd.bd = BatchDev{s->d_unused, s->d_idle, s->d_mail, s->tail, s->d_head, s->grid / 8, 0};
        sd.progress = s->d_progress;
        sd.idle_exit_ns = (long long)(s->opt.idle_exit_s * 1e9);
        cudaError_t e = launch_serve(s->form, sd, s->grid, s->threads, s->smem, s->st);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_end, s->st);
        if (e == cudaSuccess) {
            s->kernel_live = true;
            s->stats.launches += 1;
        } else {
            s->err = std::string("serve kernel launch: ") + cudaGetErrorString(e);
        }
    }
}

static void serve_thread(parrep_server_t s) {
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->quit) {
        serve_pass(s);
        s->cv.notify_all();
        s->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

static void server_free(parrep_server_t s) {
    void* dev[] = {s->d_arena, s->d_head, s->d_finished, s->d_idle, s->d_mail, s->d_unused, s->d_progress, s->d_slots};
    for (void* p : dev)
        if (p) cudaFree(p);
    void* host[] = {s->h_slot, s->done, s->tail, s->stop};
    for (void* p : host)
        if (p) cudaFreeHost(p);
    if (s->ev_end) cudaEventDestroy(s->ev_end);
    if (s->st) cudaStreamDestroy(s->st);
    if (s->cp) cudaStreamDestroy(s->cp);
}

extern "C" int parrep_server_create(const parrep_server_options* opt, parrep_server_t* out) {
    if (!out) return sfail(nullptr, PARREP_EINVAL, "out is null");
    *out = nullptr;
    parrep_server_options o;
    parrep_server_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != PARREP_FP32 && o.precision != PARREP_FP64) return sfail(nullptr, PARREP_EINVAL, "precision");
    if (o.block_threads < 0 || o.block_threads > kMaxThreads || o.block_threads % 32)
        return sfail(nullptr, PARREP_EINVAL, "block_threads must be a multiple of 32 up to 384 (0 = default)");
    const int rb = o.replicas_per_block;
    if (!(rb == 0 || rb == 32 || rb == 64 || rb == 128 || rb == 256))
        return sfail(nullptr, PARREP_EINVAL, "replicas_per_block must be 0, 32, 64, 128 or 256");
    if (o.ring < 1 || o.ring > (1 << 20)) return sfail(nullptr, PARREP_EINVAL, "ring must be 1..2^20");
    if (o.arena_bytes < (1 << 20)) return sfail(nullptr, PARREP_EINVAL, "arena_bytes below 1 MiB");
    if (o.log_cap < 1 || o.log_cap > kLogCap) return sfail(nullptr, PARREP_EINVAL, "log_cap");
    if (!(o.idle_exit_s > 0.0 && o.idle_exit_s <= 60.0)) return sfail(nullptr, PARREP_EINVAL, "idle_exit_s");
    if (!(o.wait_timeout_s > 0.0 && o.wait_timeout_s <= 3600.0))
        return sfail(nullptr, PARREP_EINVAL, "wait_timeout_s");
    if (o.f32_layout < PARREP_F32_AUTO || o.f32_layout > PARREP_F32_MIXED)
        return sfail(nullptr, PARREP_EINVAL, "f32_layout");
    // the serve kernel's form: binary64, or binary32 mixed (the default and
    // auto: each request in the layout its replica count calls for), staged
    // or direct
    const int form = o.precision == PARREP_FP64 ? kFormF64
                     : o.f32_layout == PARREP_F32_DIRECT ? kFormF32Direct
                     : o.f32_layout == PARREP_F32_AUTO || o.f32_layout == PARREP_F32_MIXED ? kFormF32Mixed
                                                         : kFormF32Staged;
    if (form == kFormF32Direct && o.block_threads > kDirectThreads)
        return sfail(nullptr, PARREP_EINVAL, "the direct layout takes at most 256 threads per block");
    const int threads = o.block_threads ? o.block_threads
                                        : (form == kFormF32Staged || form == kFormF32Mixed ? 384
                                           : form == kFormF32Direct                       ? kDirectThreads
                                                                                          : 128);
    const int RB = form == kFormF32Staged || form == kFormF32Mixed ? (rb ? rb : 32) : threads;
    if (threads < RB) return sfail(nullptr, PARREP_EINVAL, "block_threads < replicas_per_block");
    auto* s = new parrep_server_s();
    s->opt = o;
    s->form = form;
    s->threads = threads;
    s->RB = RB;
    // the direct layout keeps several blocks per SM: a smaller histogram slice
    s->smem = form == kFormF32Direct ? 64 * 1024 : 200 * 1024;
    int nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->dev);
    if (e == cudaSuccess) e = (cudaError_t)serve_attrs_form(form, &per_sm, s->smem, s->threads);
    if (e == cudaSuccess && per_sm < 1) {
        delete s;
        return sfail(nullptr, PARREP_ENOMEM, "the serve kernel does not fit on one SM");
    }
    s->grid = per_sm * nsm;
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_arena, (size_t)o.arena_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_head, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_finished, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_idle, sizeof(unsigned) * ((s->grid + 31) / 32));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_mail, sizeof(int4) * s->grid);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_unused, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_progress, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_slots, sizeof(ServeSlot) * o.ring);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->h_slot, sizeof(ServeSlot));
    if (e == cudaSuccess)
        e = cudaHostAlloc((void**)&s->done, sizeof(int) * o.ring, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void**)&s->tail, sizeof(unsigned long long), cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->stop, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_end, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(s->d_head, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_finished, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_idle, 0, sizeof(unsigned) * ((s->grid + 31) / 32));
    if (e == cudaSuccess) e = cudaMemset(s->d_mail, 0, sizeof(int4) * s->grid);
    if (e == cudaSuccess) e = cudaMemset(s->d_unused, 0x3f, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_progress, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        std::string m = std::string("parrep_server_create: ") + cudaGetErrorString(e);
        server_free(s);
        delete s;
        return sfail(nullptr, e == cudaErrorMemoryAllocation ? PARREP_ENOMEM : PARREP_ECUDA, m);
    }
    memset(s->done, 0, sizeof(int) * o.ring);
    *s->tail = 0;
    *s->stop = 0;
    s->arena.init((size_t)o.arena_bytes);
    s->slot_owner.assign(o.ring, -1);
    s->stats.arena_bytes = o.arena_bytes;
    s->stats.grid_blocks = s->grid;
    s->stats.block_threads = s->threads;
    s->th = std::thread(serve_thread, s);
    *out = s;
    return PARREP_OK;
}

extern "C" int parrep_server_submit(parrep_server_t s, const parrep_request* req, int64_t* id) {
    if (!s || !req || !id) return PARREP_EINVAL;
    std::string why;
    if (!check_network(&req->net, &req->regions, why)) return sfail(s, PARREP_EINVAL, why);
    if (req->net.kind == PARREP_GENETIC && s->form == kFormF32Staged)
        return sfail(s, PARREP_EINVAL, "the genetic switch's FP32 form needs the direct or auto layout (f32_layout)");
    if (req->n_replicas < 1 || req->n_replicas > (1ll << 30)) return sfail(s, PARREP_EINVAL, "n_replicas");
    if (!(req->t_corr >= 0.0) || !(req->t_phase >= 0.0) || !(req->t_corr < kTEndLimit * 1024) ||
        !(req->t_phase < 1e12))
        return sfail(s, PARREP_EINVAL, "t_corr / t_phase");
    if (!(req->T_end >= 0.0) || !(req->T_end < kTEndLimit)) return sfail(s, PARREP_EINVAL, "T_end");
    if (!(req->T_burn >= 0.0) || req->T_burn > req->T_end) return sfail(s, PARREP_EINVAL, "T_burn");
    if (req->thresh_mode != PARREP_THRESH_TIME && req->thresh_mode != PARREP_THRESH_STEPS)
        return sfail(s, PARREP_EINVAL, "thresh_mode");
    if (req->thresh_mode == PARREP_THRESH_STEPS &&
        (req->t_corr != (double)(long long)req->t_corr || req->t_phase != (double)(long long)req->t_phase))
        return sfail(s, PARREP_EINVAL, "STEPS mode needs integer t_corr, t_phase");
    const int g = req->fv_group;
    if (!(g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32))
        return sfail(s, PARREP_EINVAL, "fv_group");
    if (req->chunk_steps < 0 || req->chunk_steps > kMaxChunk) return sfail(s, PARREP_EINVAL, "chunk_steps");
    if (req->n_cprime < 0 || req->n_cprime > 8 || (req->n_cprime > 0 && !req->c_prime))
        return sfail(s, PARREP_EINVAL, "n_cprime must be 0..8 with c_prime");
    auto q = std::make_unique<Request>();
    q->r = *req;
    q->L = req->net.kind == PARREP_SCHLOGL ? 4 : (req->net.kind == PARREP_TOGGLE ? 6 : 8);
    q->nbins = (req->net.hist_max[0] + 1) * (req->net.hist_max[1] + 1);
    if (req->n_cprime > 0) q->cprime.assign(req->c_prime, req->c_prime + (size_t)req->n_cprime * q->L);
    q->r.c_prime = nullptr;
    q->bytes = request_bytes(*req, s->opt.log_cap);
    if (q->bytes > (size_t)s->opt.arena_bytes) return sfail(s, PARREP_EINVAL, "the request can never fit the arena");
    q->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t k = s->next_id++;
    s->reqs[k] = std::move(q);
    s->queue.push_back(k);
    s->stats.submitted += 1;
    s->stats.queued += 1;
    *id = k;
    return PARREP_OK;
}

extern "C" int parrep_server_poll(parrep_server_t s, int64_t id, int32_t* state) {
    if (!s || !state) return PARREP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, PARREP_EINVAL, "unknown request id");
    *state = it->second->state;
    return PARREP_OK;
}

extern "C" int parrep_server_wait(parrep_server_t s, int64_t id, double timeout_s) {
    if (!s) return PARREP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return sfail(s, PARREP_EINVAL, "unknown request id");
        if (it->second->state == PARREP_REQ_DONE) return PARREP_OK;
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout) {
            it = s->reqs.find(id);
            if (it != s->reqs.end() && it->second->state == PARREP_REQ_DONE) return PARREP_OK;
            return sfail(s, PARREP_ETIMEOUT, "request not done within the timeout");
        }
    }
}

extern "C" int parrep_server_result(parrep_server_t s, int64_t id, parrep_stats* stats, double* hist, int64_t len,
                                    double* fim, double* rer, double* latency_s) {
    if (!s) return PARREP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, PARREP_EINVAL, "unknown request id");
    Request& q = *it->second;
    if (q.state != PARREP_REQ_DONE) return sfail(s, PARREP_ESTATE, "request not done");
    if (hist && len != q.nbins) return sfail(s, PARREP_EINVAL, "len != n_bins");
    int rc = PARREP_OK;
    if (q.slot < 0) {
        rc = PARREP_EINVAL;  // failed admission
    } else {
        RunCtl c;
        cudaError_t e = cudaMemcpyAsync(&c, q.d_ctl_out, sizeof(RunCtl), cudaMemcpyDeviceToHost, s->cp);
        if (e == cudaSuccess && hist)
            e = cudaMemcpyAsync(hist, q.d_hist, sizeof(double) * q.nbins, cudaMemcpyDefault, s->cp);
        if (e == cudaSuccess && fim)
            e = cudaMemcpyAsync(fim, q.d_fim, sizeof(double) * q.L * q.L, cudaMemcpyDefault, s->cp);
        if (e == cudaSuccess && rer && q.r.n_cprime > 0)
            e = cudaMemcpyAsync(rer, q.d_rer, sizeof(double) * q.r.n_cprime, cudaMemcpyDefault, s->cp);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->cp);
        if (e != cudaSuccess) return sfail(s, PARREP_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
        if (stats) {
            stats_from_ctl(c, *stats);
            stats->block_threads = s->threads;
            stats->grid_blocks = c.nblk;
        }
        rc = c.status;
        s->arena.release(q.off, q.bytes);
        s->slot_owner[q.slot] = -1;
    }
    if (latency_s) *latency_s = q.t_done - q.t_submit;
    s->reqs.erase(it);
    s->stats.released += 1;
    if (rc != PARREP_OK) s->err = "the request's run failed";
    return rc;
}

extern "C" int parrep_server_stats_get(parrep_server_t s, parrep_server_stats* out) {
    if (!s || !out) return PARREP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->arena_used = (int64_t)s->arena.used();
    return PARREP_OK;
}

extern "C" void parrep_server_destroy(parrep_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.clear();  // never admitted: dropped
    }
    // admitted requests finish (the serve kernel's own waits are bounded)
    const double t_end = now_s() + 2.0 * s->opt.wait_timeout_s + 60.0;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stats.running <= 0) break;
        }
        if (now_s() > t_end) break;
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
        ((volatile int*)s->stop)[0] = 1;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaStreamSynchronize(s->st);
    server_free(s);
    delete s;
}

extern "C" const char* parrep_server_last_error(parrep_server_t s) {
    return s ? s->err.c_str() : g_server_create_error.c_str();
}
