// Host side of the C ABI declared in include/parrep.h: argument checks,
// device buffers, launch configuration and result read-back.  All arithmetic
// of the method runs in the kernels of parrep_kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "parrep.h"
#include "parrep_internal.h"
#include "parrep_handle.h"

using namespace parrep;

namespace {

thread_local std::string g_create_error;

}  // namespace

int parrep::fail(parrep_t h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int parrep::cuda_fail(parrep_t h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, PARREP_ECUDA, m);
}

#define CK(h, call)                                           \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

static cudaStream_t stream_of(parrep_t h) { return (cudaStream_t)h->opt.stream; }

extern "C" void parrep_default_options(parrep_options* o) {
    memset(o, 0, sizeof(*o));
    o->thresh_mode = PARREP_THRESH_TIME;
    o->precision = PARREP_FP64;
    o->fv_group = 32;
    o->block_threads = 0;
    o->chunk_steps = 0;
    o->debug_stall_barrier = -1;
    o->serial_stages = 0;
    o->max_blocks = 0;
    o->T_burn = 0.0;
    o->wait_timeout_s = 10.0;
    o->stream = nullptr;
}

int parrep::check_network(const parrep_network* net, const parrep_regions* reg, std::string& why) {
    if (!net || !reg) { why = "null network or regions"; return 0; }
    if (net->kind != PARREP_SCHLOGL && net->kind != PARREP_TOGGLE && net->kind != PARREP_GENETIC) {
        why = "unknown network kind";
        return 0;
    }
    const int nsp = net->kind == PARREP_SCHLOGL ? 1 : 2;
    if (net->n_species != nsp) { why = "n_species does not match the kind"; return 0; }
    if (net->hist_max[0] < 0 || net->hist_max[1] < 0 || (nsp == 1 && net->hist_max[1] != 0)) {
        why = "bad hist_max";
        return 0;
    }
    const long long nb = (long long)(net->hist_max[0] + 1) * (net->hist_max[1] + 1);
    if (nb > (1ll << 24)) { why = "more than 2^24 histogram bins"; return 0; }
    const int L = nsp == 1 ? 4 : (net->kind == PARREP_TOGGLE ? 6 : 8);
    for (int i = 0; i < L; ++i)
        if (!std::isfinite(net->c[i])) { why = "non-finite rate constant"; return 0; }
    if (net->kind == PARREP_GENETIC) {
        for (int i = 0; i < 8; ++i)
            if (!(net->c[i] >= 0.0)) { why = "genetic switch constants must be >= 0"; return 0; }
        if (!(net->c[7] > 0.0)) { why = "genetic switch needs D > 0"; return 0; }
    } else if (nsp == 1) {
        for (int i = 0; i < 4; ++i)
            if (!(net->c[i] >= 0.0) || !(net->s[i] >= 0.0) || !std::isfinite(net->s[i])) {
                why = "Schloegl constants must be finite and >= 0";
                return 0;
            }
        if (!(net->c[2] * net->s[2] > 0.0)) { why = "Schloegl needs c3*s3 > 0 (a0 > 0 everywhere)"; return 0; }
    } else {
        if (!(net->c[0] > 0.0) || !(net->c[3] > 0.0) || !(net->c[2] >= 0.0) || !(net->c[5] >= 0.0)) {
            why = "toggle rates must be positive";
            return 0;
        }
    }
    if (nsp == 2 && (net->hist_max[0] > 32767 || net->hist_max[1] > 32767)) {
        why = "two-species hist_max must be <= 32767 per species";
        return 0;
    }
    if (reg->n < 1 || reg->n > 4) { why = "regions: n must be 1..4"; return 0; }
    if (net->x0_uniform_hi < 0) { why = "x0_uniform_hi < 0"; return 0; }
    if (net->x0_uniform_hi > 0) {
        if (net->x0_uniform_hi > net->hist_max[0] || (nsp == 2 && net->x0_uniform_hi > net->hist_max[1])) {
            why = "x0_uniform_hi beyond hist_max";
            return 0;
        }
    } else {
        if (net->x0[0] < 0 || net->x0[0] > net->hist_max[0] ||
            (nsp == 2 && (net->x0[1] < 0 || net->x0[1] > net->hist_max[1]))) {
            why = "x0 outside [0, hist_max]";
            return 0;
        }
    }
    return 1;
}

// Host-built tables (toggle production rates, their log-derivatives in the
// Hill exponent) and the network constants as the kernels read them.
void parrep::build_net(const parrep_network* net, const parrep_regions* reg, NetDev& nd,
                      std::vector<double>& pU, std::vector<double>& pV, std::vector<double>& gU,
                      std::vector<double>& gV) {
    memset(&nd, 0, sizeof(nd));
    nd.kind = net->kind;
    nd.nsp = net->n_species;
    nd.hist_max0 = net->hist_max[0];
    nd.hist_max1 = net->hist_max[1];
    nd.ystride = net->hist_max[1] + 1;
    nd.nbins = (net->hist_max[0] + 1) * (net->hist_max[1] + 1);
    nd.nreg = reg->n;
    for (int i = 0; i < reg->n; ++i) {
        nd.ra0[i] = reg->a[i][0];
        nd.ra1[i] = net->n_species > 1 ? reg->a[i][1] : 0;
        nd.rb[i] = reg->b[i];
    }
    for (int i = 0; i < 5; ++i) {
        nd.wlo[i] = 1;
        nd.whi[i] = 0;
    }
    if (net->n_species == 1) {
        for (int x = 0; x <= net->hist_max[0]; ++x) {
            int rg = reg->n;
            for (int i = 0; i < reg->n; ++i)
                if ((long long)reg->a[i][0] * x < reg->b[i]) {
                    rg = i;
                    break;
                }
            if (nd.wlo[rg] > nd.whi[rg]) nd.wlo[rg] = x;
            nd.whi[rg] = x;
        }
    }
    if (net->kind == PARREP_GENETIC) {
        // a, gamma, gamma b; the switching rates F(p), G(p) as tables over p
        const double* c = net->c;
        nd.A[0] = c[0];
        nd.A[1] = c[2];
        nd.A[2] = c[2] * c[1];
        for (int j = 0; j < 3; ++j) nd.Af[j] = (float)nd.A[j];  // the binary32 form's constants
        pU.resize(net->hist_max[1] + 1);
        pV.resize(net->hist_max[1] + 1);
        for (int v = 0; v <= net->hist_max[1]; ++v) {
            const double p = (double)v;
            const double hh = p * p / (p * p + c[7] * c[7]);
            pU[v] = c[3] + (c[4] - c[3]) * hh;
            pV[v] = c[6] - (c[6] - c[5]) * hh;
        }
    } else if (net->kind == PARREP_SCHLOGL) {
        for (int j = 0; j < 4; ++j) {
            nd.A[j] = net->c[j] * net->s[j];
            nd.Af[j] = (float)nd.A[j];
        }
    } else {
        nd.dU = net->c[2];
        nd.dV = net->c[5];
        nd.dUf = (float)net->c[2];
        nd.dVf = (float)net->c[5];
        pU.resize(net->hist_max[1] + 1);
        gU.resize(net->hist_max[1] + 1);
        for (int v = 0; v <= net->hist_max[1]; ++v) {
            const double p = pow((double)v, net->c[1]);
            pU[v] = net->c[0] / (1.0 + p);
            gU[v] = v > 0 ? -p * log((double)v) / (1.0 + p) : 0.0;
        }
        pV.resize(net->hist_max[0] + 1);
        gV.resize(net->hist_max[0] + 1);
        for (int u = 0; u <= net->hist_max[0]; ++u) {
            const double p = pow((double)u, net->c[4]);
            pV[u] = net->c[3] / (1.0 + p);
            gV[u] = u > 0 ? -p * log((double)u) / (1.0 + p) : 0.0;
        }
    }
}

template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& v) {
    if (v.empty()) { *dst = nullptr; return cudaSuccess; }
    cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_all(parrep_t h) {
    void* ptrs[] = {h->d_prodU_d, h->d_prodV_d, h->d_prodU_f, h->d_prodV_f, h->d_gradU_n, h->d_gradV_n,
                    h->d_c, h->d_s, h->d_ctl, h->d_hist_pre, h->d_hist_post, h->d_step_sum, h->d_tau_at,
                    h->d_log, h->d_out, h->d_out2, h->d_fim, h->d_rer, h->d_cprime, h->d_xstate};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
}

extern "C" int parrep_create(const parrep_network* net, int64_t n_replicas, const parrep_regions* reg,
                             double t_corr, double t_phase, parrep_t* out) {
    if (!out) return fail(nullptr, PARREP_EINVAL, "out is null");
    *out = nullptr;
    std::string why;
    if (!check_network(net, reg, why)) return fail(nullptr, PARREP_EINVAL, why);
    if (n_replicas < 1 || n_replicas > (1ll << 30)) return fail(nullptr, PARREP_EINVAL, "n_replicas outside [1, 2^30]");
    if (!(t_corr >= 0.0) || !(t_phase >= 0.0) || !(t_corr < kTEndLimit * 1024) || !(t_phase < 1e12))
        return fail(nullptr, PARREP_EINVAL, "t_corr / t_phase must be finite and >= 0");
    parrep_s* h = new parrep_s();
    h->net = *net;
    h->reg = *reg;
    h->R = n_replicas;
    h->t_corr = t_corr;
    h->t_phase = t_phase;
    parrep_default_options(&h->opt);
    h->nbins = (net->hist_max[0] + 1) * (net->hist_max[1] + 1);
    h->L = net->kind == PARREP_SCHLOGL ? 4 : (net->kind == PARREP_TOGGLE ? 6 : 8);
    std::vector<double> pU, pV, gU, gV;
    build_net(net, reg, h->nd, pU, pV, gU, gV);
    cudaError_t e = cudaSuccess;
    std::vector<float> pUf(pU.begin(), pU.end()), pVf(pV.begin(), pV.end());
    for (size_t i = 0; i < pU.size(); ++i) pUf[i] = (float)pU[i];
    for (size_t i = 0; i < pV.size(); ++i) pVf[i] = (float)pV[i];
    std::vector<double> cv(net->c, net->c + 8), sv(net->s, net->s + 4);
#define TRY(x)                      \
    do {                            \
        e = (x);                    \
        if (e != cudaSuccess) goto bad; \
    } while (0)
    TRY(upload(&h->d_prodU_d, pU));
    TRY(upload(&h->d_prodV_d, pV));
    TRY(upload(&h->d_prodU_f, pUf));
    TRY(upload(&h->d_prodV_f, pVf));
    TRY(upload(&h->d_gradU_n, gU));
    TRY(upload(&h->d_gradV_n, gV));
    TRY(upload(&h->d_c, cv));
    TRY(upload(&h->d_s, sv));
    TRY(cudaMalloc((void**)&h->d_ctl, sizeof(RunCtl)));
    TRY(cudaMalloc((void**)&h->d_hist_pre, sizeof(unsigned long long) * h->nbins));
    TRY(cudaMalloc((void**)&h->d_hist_post, sizeof(unsigned long long) * h->nbins));
    TRY(cudaMalloc((void**)&h->d_step_sum, sizeof(unsigned long long) * kMaxChunk));
    TRY(cudaMalloc((void**)&h->d_tau_at, sizeof(unsigned long long) * 2 * (size_t)n_replicas));
    TRY(cudaMalloc((void**)&h->d_log, sizeof(CycleRecDev) * kLogCap));
    TRY(cudaMalloc((void**)&h->d_xstate, sizeof(int2) * 3 * (size_t)n_replicas));
    TRY(cudaMalloc((void**)&h->d_out, sizeof(double) * h->nbins));
    TRY(cudaMalloc((void**)&h->d_out2, sizeof(double) * h->nbins));
    TRY(cudaMalloc((void**)&h->d_fim, sizeof(double) * 64));
    TRY(cudaMalloc((void**)&h->d_rer, sizeof(double) * 8));
    TRY(cudaMalloc((void**)&h->d_cprime, sizeof(double) * 8 * 8));
    TRY(cudaEventCreate(&h->ev0));
    TRY(cudaEventCreate(&h->ev1));
    TRY(cudaMemset(h->d_hist_pre, 0, sizeof(unsigned long long) * h->nbins));
    TRY(cudaMemset(h->d_hist_post, 0, sizeof(unsigned long long) * h->nbins));
    h->nd.prodU_d = h->d_prodU_d;
    h->nd.prodV_d = h->d_prodV_d;
    h->nd.prodU_f = h->d_prodU_f;
    h->nd.prodV_f = h->d_prodV_f;
#undef TRY
    *out = h;
    return PARREP_OK;
bad : {
    std::string m = std::string("parrep_create: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? PARREP_ENOMEM : PARREP_ECUDA, m);
}
}

extern "C" int parrep_set_options(parrep_t h, const parrep_options* o) {
    if (!h) return PARREP_EINVAL;
    parrep_options d;
    parrep_default_options(&d);
    if (!o) { h->opt = d; return PARREP_OK; }
    if (o->thresh_mode != PARREP_THRESH_TIME && o->thresh_mode != PARREP_THRESH_STEPS)
        return fail(h, PARREP_EINVAL, "thresh_mode");
    if (o->precision != PARREP_FP64 && o->precision != PARREP_FP32) return fail(h, PARREP_EINVAL, "precision");
    const int g = o->fv_group;
    if (!(g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32))
        return fail(h, PARREP_EINVAL, "fv_group must be 1, 2, 4, 8, 16 or 32");
    if (o->block_threads < 0 || o->block_threads > kMaxThreads || (o->block_threads % 32) != 0)
        return fail(h, PARREP_EINVAL, "block_threads must be a multiple of 32 up to 384 (0 = auto)");
    if (o->chunk_steps < 0 || o->chunk_steps > kMaxChunk) return fail(h, PARREP_EINVAL, "chunk_steps");
    if (o->max_blocks < 0) return fail(h, PARREP_EINVAL, "max_blocks must be >= 0");
    if (o->f32_layout < PARREP_F32_AUTO || o->f32_layout > PARREP_F32_MIXED)
        return fail(h, PARREP_EINVAL, "f32_layout must be PARREP_F32_AUTO, _STAGED, _DIRECT or _MIXED");
    if (h->net.kind == PARREP_GENETIC && o->precision == PARREP_FP32 && o->f32_layout == PARREP_F32_STAGED)
        return fail(h, PARREP_EINVAL, "the genetic switch's FP32 form runs in the direct layout only");
    if (!(o->T_burn >= 0.0) || !(o->T_burn < kTEndLimit)) return fail(h, PARREP_EINVAL, "T_burn");
    if (!(o->wait_timeout_s > 0.0) || !(o->wait_timeout_s <= 3600.0)) return fail(h, PARREP_EINVAL, "wait_timeout_s");
    if (o->thresh_mode == PARREP_THRESH_STEPS) {
        if (h->t_corr != floor(h->t_corr) || h->t_phase != floor(h->t_phase) || h->t_phase > 4294967294.0)
            return fail(h, PARREP_EINVAL, "STEPS mode needs integer t_corr, t_phase (t_phase < 2^32-1)");
    } else if (!(h->t_corr < kTEndLimit)) {
        return fail(h, PARREP_EINVAL, "TIME mode needs t_corr < 2^23");
    }
    h->opt = *o;
    return PARREP_OK;
}

int parrep::align16(int x) { return (x + 15) & ~15; }

int parrep::fast_layout(parrep_t h, int RB, int threads, int with_hist, int pipelined, Plan& pl) {
    const int B = staged_sub_chunk(RB);
    const int nbuf = pipelined ? 3 : 1, ntr = pipelined ? 2 : 1;
    pl.pipelined = pipelined;
    int off = 0;
    pl.use_smem_hist = with_hist;
    pl.off_limbs = -1;
    if (with_hist) {
        off += align16(h->nbins * 8);
        pl.off_limbs = off;
        off += align16(h->nbins * 8);  // two 32-bit limbs per bin
    }
    pl.off_tab = -1;
    pl.off_inv = -1;
    pl.off_thr = -1;
    if (h->net.kind == PARREP_SCHLOGL) {
        // per state RN(1/a0) and the choice thresholds (int4, kThrPad entries
        // beyond each end), for ranges up to about 4000 states
        const int tb = (h->net.hist_max[0] + 1 + 2 * kThrPad) * 16;
        if (tb <= 64 * 1024) {
            pl.off_inv = off;
            off += align16((h->net.hist_max[0] + 1) * 4);
            pl.off_thr = off;
            off += align16(tb);
        }
    } else {
        pl.off_tab = off;
        off += align16((h->net.hist_max[0] + 1 + h->net.hist_max[1] + 1) * 4);
    }
    pl.off_buf = off;
    off += nbuf * B * RB * 8;
    pl.off_trace = off;
    off += ntr * B * RB * 4;
    pl.off_live = off;
    off += RB * 4;
    pl.off_nvalid = off;
    off += ntr * RB * 4;
    pl.off_rng = off;
    off += 48;  // three rectangles of touched states (12 ints)
    pl.off_decp = off;  // decorrelation rounds of min(4 x threads, B x RB) steps
    off += (4 * threads < B * RB ? 4 * threads : B * RB) * 8;
    pl.B = B;
    pl.RB = RB;
    int l = 0;
    while ((1 << l) < RB) ++l;
    pl.log2RB = l;
    return off;
}

// The kernel form of a handle's runs: binary64; or, in the FP32 form, the
// staged layout (each owner thread's chain fed by helper warps) or the direct
// one (one thread per replica): as the option asks, else direct for the
// genetic switch (whose six channels the staged chain does not take) and from
// kDirectAutoReplicas replicas on (measured: 2.2x faster at 16384 replicas,
// 2-3.4x at 65536), staged below (10x faster at 4096).
int parrep::f32_form(parrep_t h) {
    if (h->opt.precision != PARREP_FP32) return kFormF64;
    if (h->opt.f32_layout == PARREP_F32_STAGED) return kFormF32Staged;
    if (h->opt.f32_layout == PARREP_F32_DIRECT || h->net.kind == PARREP_GENETIC) return kFormF32Direct;
    return h->R >= kDirectAutoReplicas ? kFormF32Direct : kFormF32Staged;
}

static int plan_launch(parrep_t h, Plan& pl) {
    int dev = 0, nsm = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int prec = h->opt.precision, kind = h->net.kind;
    memset(&pl, 0, sizeof(pl));
    int per_sm = 0;
    const int form = f32_form(h);
    if (form != kFormF32Staged) {
        // one thread per replica (binary64, or binary32 direct)
        const int cap = form == kFormF32Direct ? kDirectThreads : kMaxThreads;
        int threads = h->opt.block_threads > 0 ? h->opt.block_threads : (form == kFormF32Direct ? kDirectThreads : 128);
        if (threads > cap) threads = cap;
        if ((long long)threads > ((h->R + 31) / 32) * 32) threads = (int)(((h->R + 31) / 32) * 32);
        pl.form = form;
        pl.threads = threads;
        pl.RB = threads;
        pl.grid = (int)((h->R + threads - 1) / threads);
        pl.S = h->opt.chunk_steps > 0 ? h->opt.chunk_steps : default_chunk(false, h->R);
        pl.off_tab = pl.off_buf = pl.off_trace = pl.off_live = pl.off_nvalid = -1;
        pl.off_limbs = pl.off_inv = pl.off_rng = pl.off_decp = pl.off_thr = -1;
        pl.pipelined = 0;
        for (int with_hist = 1; with_hist >= 0; --with_hist) {
            if (with_hist && h->nbins * 8 > (form == kFormF32Direct ? kDirectSmemHistLimit : kSmemHistLimit)) continue;
            pl.use_smem_hist = with_hist;
            pl.smem = with_hist ? h->nbins * 8 : 0;
            int ea = kernel_attrs_form(form, kind, &per_sm, pl.smem, threads);
            if (ea != 0) return cuda_fail(h, (cudaError_t)ea, "kernel attributes");
            if (per_sm < 1) continue;
            // more replica groups than co-resident blocks: blocks take several
            if ((long long)per_sm * nsm < pl.grid) pl.grid = per_sm * nsm;
            if (h->opt.max_blocks > 0 && pl.grid > h->opt.max_blocks) pl.grid = h->opt.max_blocks;
            return PARREP_OK;
        }
        return fail(h, PARREP_ENOMEM, "the run kernel does not fit on one SM");
    }
    const int T = h->opt.block_threads > 0 ? h->opt.block_threads : 384;
    // the smallest RB whose grid is co-resident; if none is, RB = 32 on a
    // full co-resident grid, each block taking several groups of replicas
    for (int pass = 0; pass < 2; ++pass)
    for (int RB = 32; RB <= (pass ? 32 : 256); RB *= 2) {  // RB <= 256 keeps threads <= kMaxThreads
        const int threads = RB > T ? RB : T;
        const long long grid = (h->R + RB - 1) / RB;
        for (int cfg = 3; cfg >= 0; --cfg) {
            // prefer the warp-specialised pipeline (needs >= 2 helper warps),
            // then the shared-memory histogram
            const int pipe = (cfg & 2) && threads - RB >= 64 && !h->opt.serial_stages;
            const int with_hist = cfg & 1;
            if ((cfg & 2) && !pipe) continue;
            const int smem = fast_layout(h, RB, threads, with_hist, pipe, pl);
            if (smem > 200 * 1024) continue;
            pl.form = kFormF32Staged;
            int ea = kernel_attrs_form(kFormF32Staged, kind, &per_sm, smem, threads);
            if (ea != 0) return cuda_fail(h, (cudaError_t)ea, "kernel attributes");
            if (per_sm < 1) continue;
            if ((long long)per_sm * nsm >= grid || pass == 1) {
                pl.threads = threads;
                pl.grid = (long long)per_sm * nsm >= grid ? (int)grid : per_sm * nsm;
                if (h->opt.max_blocks > 0 && pl.grid > h->opt.max_blocks) pl.grid = h->opt.max_blocks;
                pl.smem = smem;
                const int S = h->opt.chunk_steps > 0 ? h->opt.chunk_steps : default_chunk(true, h->R);
                pl.S = ((S + pl.B - 1) / pl.B) * pl.B;
                return PARREP_OK;
            }
        }
    }
    return fail(h, PARREP_ENOMEM, "the run kernel does not fit on one SM");
}

// Checks of parrep_run's arguments against the handle's options.
int parrep::run_checks(parrep_t h, double T_end) {
    h->has_run = false;
    if (!(T_end >= 0.0) || !(T_end < kTEndLimit)) return fail(h, PARREP_EINVAL, "T_end must be in [0, 2^23)");
    if (h->opt.T_burn > T_end) return fail(h, PARREP_EINVAL, "T_burn > T_end");
    if (h->opt.thresh_mode == PARREP_THRESH_STEPS &&
        (h->t_corr != floor(h->t_corr) || h->t_phase != floor(h->t_phase)))
        return fail(h, PARREP_EINVAL, "STEPS mode needs integer t_corr, t_phase");
    return PARREP_OK;
}

// The kernel parameters of one run of h with launch plan pl.
int parrep::run_params(parrep_t h, double T_end, uint64_t seed, const Plan& pl, RunParams& p) {
    const int grid = pl.grid, S = pl.S;
    if (S > kMaxChunk) return fail(h, PARREP_EINVAL, "chunk_steps too large");
    memset(&p, 0, sizeof(p));
    p.net = h->nd;
    p.prec = h->opt.precision;
    p.form = pl.form;
    p.thresh = h->opt.thresh_mode;
    p.R = (int)h->R;
    p.G = h->opt.fv_group;
    p.S = S;
    p.use_smem_hist = pl.use_smem_hist;
    p.RB = pl.RB;
    p.log2RB = pl.log2RB;
    p.B = pl.B;
    p.off_tab = pl.off_tab;
    p.off_buf = pl.off_buf;
    p.off_trace = pl.off_trace;
    p.off_live = pl.off_live;
    p.off_nvalid = pl.off_nvalid;
    p.off_limbs = pl.off_limbs;
    p.off_inv = pl.off_inv;
    p.off_rng = pl.off_rng;
    p.off_decp = pl.off_decp;
    p.off_thr = pl.off_thr;
    p.pipelined = pl.pipelined;
    if (p.thresh == PARREP_THRESH_STEPS) {
        p.n_c = (long long)h->t_corr;
        p.n_p = (long long)h->t_phase;
    } else {
        p.q_tcorr = (unsigned long long)llrint(h->t_corr * kQScale);
        p.t_phase = h->t_phase;
    }
    p.q_Tend = (unsigned long long)llrint(T_end * kQScale);
    p.q_Tburn = (unsigned long long)llrint(h->opt.T_burn * kQScale);
    p.seed = seed;
    p.x00 = h->net.x0[0];
    p.x01 = h->net.n_species > 1 ? h->net.x0[1] : 0;
    p.x0_hi = h->net.x0_uniform_hi;
    p.ctl = h->d_ctl;
    p.hist_pre = h->d_hist_pre;
    p.hist_post = h->d_hist_post;
    p.step_sum = h->d_step_sum;
    p.tau_at = h->d_tau_at;
    p.nblk = grid;
    p.xs = h->d_xstate;
    p.xk = h->d_xstate + h->R;
    p.xe = h->d_xstate + 2 * h->R;
    p.log = h->d_log;
    p.log_cap = kLogCap;
    p.timeout_ns = (long long)(h->opt.wait_timeout_s * 1e9);
    p.stall_barrier = h->opt.debug_stall_barrier;
    p.progress = &h->d_ctl->progress;
    return PARREP_OK;
}

// Statistics of a finished run from its control block c.
void parrep::stats_from_ctl(const RunCtl& c, parrep_stats& s) {
    memset(&s, 0, sizeof(s));
    s.T_s = (double)c.Ts * kQInv;
    s.events_decorr = (int64_t)c.ev_decorr;
    s.events_dephase = (int64_t)c.ev_dephase;
    s.events_parallel_useful = (int64_t)c.ev_useful;
    s.events_parallel_executed = (int64_t)c.ev_par_exec;
    s.events_replay = (int64_t)c.ev_replay;
    s.cycles = (int64_t)c.cycles;
    s.escapes = (int64_t)c.escapes;
    s.chunks = (int64_t)c.chunks;
    s.special_chunks = (int64_t)c.special;
    s.x0[0] = c.x00;
    s.x0[1] = c.x01;
    s.x_final[0] = c.xt0;
    s.x_final[1] = c.xt1;
    s.status = c.status;
    for (int i = 0; i < 12; ++i) s.phase_cycles[i] = (double)c.phase_cycles[i];
}

int parrep::run_finish(parrep_t h, const RunCtl& c, double T_end, const Plan& pl, float ms) {
    h->h_ctl = c;
    parrep_stats& s = h->stats;
    stats_from_ctl(c, s);
    s.grid_blocks = pl.grid;
    s.block_threads = pl.threads;
    s.chunk_steps = pl.S;
    s.kernel_ms = ms;
    h->T_end = T_end;
    h->T_burn = h->opt.T_burn;
    if (c.status != 0) {
        const char* what = c.status == PARREP_ERANGE     ? "a state left [0, hist_max] or a step counter overflowed"
                           : c.status == PARREP_ETIMEOUT ? "a device wait timed out without progress"
                           : c.status == PARREP_EINVAL   ? "invalid initial state"
                                                         : "device error";
        return fail(h, c.status, what);
    }
    h->has_run = true;
    return PARREP_OK;
}

extern "C" int parrep_run(parrep_t h, double T_end, uint64_t seed) {
    if (!h) return PARREP_EINVAL;
    int rc = run_checks(h, T_end);
    if (rc != PARREP_OK) return rc;
    Plan pl;
    rc = plan_launch(h, pl);
    if (rc != PARREP_OK) return rc;
    RunParams p;
    rc = run_params(h, T_end, seed, pl, p);
    if (rc != PARREP_OK) return rc;
    cudaStream_t st = stream_of(h);
    CK(h, cudaMemsetAsync(h->d_ctl, 0, sizeof(RunCtl), st));
    CK(h, cudaMemsetAsync(h->d_hist_pre, 0, sizeof(unsigned long long) * h->nbins, st));
    CK(h, cudaMemsetAsync(h->d_hist_post, 0, sizeof(unsigned long long) * h->nbins, st));
    CK(h, cudaEventRecord(h->ev0, st));
    CK(h, launch_run(p, pl.grid, pl.threads, pl.smem, st));
    CK(h, cudaEventRecord(h->ev1, st));
    RunCtl c;
    CK(h, cudaMemcpyAsync(&c, h->d_ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    return run_finish(h, c, T_end, pl, ms);
}

extern "C" int64_t parrep_n_bins(parrep_t h) { return h ? (int64_t)h->nbins : 0; }

extern "C" int parrep_histogram(parrep_t h, double* out, int64_t len) {
    if (!h || !out) return PARREP_EINVAL;
    if (!h->has_run) return fail(h, PARREP_ESTATE, "no completed run");
    if (len != h->nbins) return fail(h, PARREP_EINVAL, "len != n_bins");
    const double Ts = h->stats.T_s;
    cudaStream_t st = stream_of(h);
    CK(h, launch_hist_normalise(h->d_hist_pre, h->d_hist_post, h->nbins, Ts > 0 ? 1.0 / Ts : 0.0, nullptr, nullptr,
                                h->d_out, st));
    CK(h, cudaMemcpyAsync(out, h->d_out, sizeof(double) * h->nbins, cudaMemcpyDefault, st));
    CK(h, cudaStreamSynchronize(st));
    return PARREP_OK;
}

extern "C" int parrep_histogram_raw(parrep_t h, double* pre, double* post, int64_t len) {
    if (!h) return PARREP_EINVAL;
    if (!h->has_run) return fail(h, PARREP_ESTATE, "no completed run");
    if (len != h->nbins) return fail(h, PARREP_EINVAL, "len != n_bins");
    cudaStream_t st = stream_of(h);
    CK(h, launch_hist_normalise(h->d_hist_pre, h->d_hist_post, h->nbins, 0.0, h->d_out, h->d_out2, nullptr, st));
    if (pre) CK(h, cudaMemcpyAsync(pre, h->d_out, sizeof(double) * h->nbins, cudaMemcpyDefault, st));
    if (post) CK(h, cudaMemcpyAsync(post, h->d_out2, sizeof(double) * h->nbins, cudaMemcpyDefault, st));
    CK(h, cudaStreamSynchronize(st));
    return PARREP_OK;
}

static int contract(parrep_t h, const double* cprime, int n, double* fim_host, double* rer_host) {
    cudaStream_t st = stream_of(h);
    CK(h, cudaMemsetAsync(h->d_fim, 0, sizeof(double) * 64, st));
    CK(h, cudaMemsetAsync(h->d_rer, 0, sizeof(double) * 8, st));
    if (n > 0)
        CK(h, cudaMemcpyAsync(h->d_cprime, cprime, sizeof(double) * n * h->L, cudaMemcpyHostToDevice, st));
    CK(h, launch_fim_rer(h->nd, h->d_c, h->d_s, h->d_hist_post, h->d_gradU_n, h->d_gradV_n, h->d_cprime, n,
                         h->d_fim, h->d_rer, st));
    if (fim_host) CK(h, cudaMemcpyAsync(fim_host, h->d_fim, sizeof(double) * 64, cudaMemcpyDeviceToHost, st));
    if (rer_host) CK(h, cudaMemcpyAsync(rer_host, h->d_rer, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    return PARREP_OK;
}

extern "C" int parrep_fim(parrep_t h, double* out, int32_t len) {
    if (!h || !out) return PARREP_EINVAL;
    if (!h->has_run) return fail(h, PARREP_ESTATE, "no completed run");
    if (len != h->L * h->L) return fail(h, PARREP_EINVAL, "len != l*l");
    const double span = h->stats.T_s - h->T_burn;
    if (!(span > 0.0)) return fail(h, PARREP_ESTATE, "empty window [T_burn, T_end]");
    double buf[64];
    int rc = contract(h, nullptr, 0, buf, nullptr);
    if (rc) return rc;
    double res[64];
    for (int i = 0; i < h->L * h->L; ++i) res[i] = buf[i] / span;
    CK(h, cudaMemcpy(out, res, sizeof(double) * h->L * h->L, cudaMemcpyDefault));
    return PARREP_OK;
}

extern "C" int parrep_rer(parrep_t h, const double* c_prime, int32_t n, double* out) {
    if (!h || !out || (n > 0 && !c_prime) || n < 0) return PARREP_EINVAL;
    if (!h->has_run) return fail(h, PARREP_ESTATE, "no completed run");
    const double span = h->stats.T_s - h->T_burn;
    if (!(span > 0.0)) return fail(h, PARREP_ESTATE, "empty window [T_burn, T_end]");
    std::vector<double> res(n);
    for (int k0 = 0; k0 < n; k0 += 8) {
        const int m = n - k0 < 8 ? n - k0 : 8;
        for (int k = 0; k < m; ++k)
            for (int i = 0; i < h->L; ++i)
                // every perturbed constant > 0 (the toggle's Hill exponents excepted),
                // so that lambda' > 0 wherever lambda > 0
                if (!(c_prime[(k0 + k) * h->L + i] > 0.0) &&
                    !(h->net.kind == PARREP_TOGGLE && (i == 1 || i == 4)))
                    return fail(h, PARREP_EINVAL, "perturbed rate constants must be > 0");
        double buf[8];
        int rc = contract(h, c_prime + (size_t)k0 * h->L, m, nullptr, buf);
        if (rc) return rc;
        for (int k = 0; k < m; ++k) res[k0 + k] = buf[k] / span;
    }
    if (n > 0) CK(h, cudaMemcpy(out, res.data(), sizeof(double) * n, cudaMemcpyDefault));
    return PARREP_OK;
}

extern "C" int parrep_stats_get(parrep_t h, parrep_stats* out) {
    if (!h || !out) return PARREP_EINVAL;
    *out = h->stats;
    return PARREP_OK;
}

extern "C" int parrep_cycle_log(parrep_t h, parrep_cycle* out, int64_t cap, int64_t* n_out) {
    if (!h || (!out && cap > 0) || cap < 0) return PARREP_EINVAL;
    if (!h->has_run && h->h_ctl.log_n == 0) return fail(h, PARREP_ESTATE, "no run");
    const long long n = h->h_ctl.log_n;
    if (n_out) *n_out = n;
    long long m = n < cap ? n : cap;
    if (m > kLogCap) m = kLogCap;
    if (m <= 0) return PARREP_OK;
    std::vector<CycleRecDev> buf(m);
    CK(h, cudaMemcpy(buf.data(), h->d_log, sizeof(CycleRecDev) * m, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < m; ++i) {
        parrep_cycle& c = out[i];
        const CycleRecDev& d = buf[i];
        c.cycle = d.cycle;
        c.W = d.W;
        c.ended = d.ended;
        c.decorr_steps = d.decorr_steps;
        c.dephase_steps = d.dephase_steps;
        c.n_star = d.n_star;
        c.k = d.k;
        c.x_tilde[0] = d.xt0;
        c.x_tilde[1] = d.xt1;
        c.T_s = (double)d.Ts * kQInv;
    }
    return PARREP_OK;
}

extern "C" int parrep_dephase(parrep_t h, const int32_t* x_tilde, int32_t W, uint32_t cycle, uint64_t seed,
                              int32_t* out_states) {
    if (!h || !x_tilde || !out_states) return PARREP_EINVAL;
    const int x0 = x_tilde[0], x1 = h->net.n_species > 1 ? x_tilde[1] : 0;
    if (x0 < 0 || x0 > h->net.hist_max[0] || x1 < 0 || x1 > h->net.hist_max[1])
        return fail(h, PARREP_EINVAL, "x_tilde outside [0, hist_max]");
    long long np;
    if (h->opt.thresh_mode == PARREP_THRESH_STEPS) {
        np = (long long)h->t_phase;
    } else {
        // a0 at X~ in binary64, the same expression as the kernels'
        double l0 = 0.0, l1 = 0.0, l2 = 0.0, l3 = 0.0;
        const NetDev& N = h->nd;
        if (N.kind == PARREP_SCHLOGL) {
            const double xd = (double)x0;
            const double a = xd * (xd - 1.0);
            const double b = a * (xd - 2.0);
            l0 = N.A[0] * a;
            l1 = N.A[1] * b;
            l2 = N.A[2];
            l3 = N.A[3] * xd;
        } else if (N.kind != PARREP_GENETIC) {
            CK(h, cudaMemcpy(&l0, h->d_prodU_d + x1, sizeof(double), cudaMemcpyDeviceToHost));
            CK(h, cudaMemcpy(&l1, h->d_prodV_d + x0, sizeof(double), cudaMemcpyDeviceToHost));
            l2 = N.dU * (double)x0;
            l3 = N.dV * (double)x1;
        }
        double a0 = ((l0 + l1) + l2) + l3;
        if (N.kind == PARREP_GENETIC) {
            // six channels: a xi, gamma m, gamma b m, p, F(p)(1 - xi), G(p) xi
            double F, G;
            CK(h, cudaMemcpy(&F, h->d_prodU_d + x1, sizeof(double), cudaMemcpyDeviceToHost));
            CK(h, cudaMemcpy(&G, h->d_prodV_d + x1, sizeof(double), cudaMemcpyDeviceToHost));
            const double xi = (double)(x0 & 1), m = (double)(x0 >> 1);
            a0 = ((((N.A[0] * xi + N.A[1] * m) + N.A[2] * m) + (double)x1) + F * (1.0 - xi)) + G * xi;
        }
        const double n = ceil(h->t_phase * a0);
        if (!(n < 4294967295.0)) return fail(h, PARREP_ERANGE, "dephasing step count >= 2^32-1");
        np = (long long)n;
    }
    RunParams p;
    memset(&p, 0, sizeof(p));
    p.net = h->nd;
    p.prec = h->opt.precision;
    p.R = (int)h->R;
    p.G = h->opt.fv_group;
    p.RB = 128;
    p.seed = seed;
    p.ctl = h->d_ctl;
    cudaStream_t st = stream_of(h);
    int* d_states = nullptr;
    CK(h, cudaMalloc((void**)&d_states, sizeof(int) * 2 * h->R));
    CK(h, cudaMemsetAsync(h->d_ctl, 0, sizeof(RunCtl), st));
    const int threads = 128;
    const int grid = (int)((h->R + threads - 1) / threads);
    cudaError_t e = launch_dephase(p, x0, x1, W, cycle, np, d_states, grid, threads, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_states, d_states, sizeof(int) * 2 * h->R, cudaMemcpyDefault, st);
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &h->d_ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_states);
    if (e != cudaSuccess) return cuda_fail(h, e, "dephase");
    if (status) return fail(h, status, "a dephasing state left [0, hist_max]");
    return PARREP_OK;
}

extern "C" void parrep_destroy(parrep_t h) {
    if (!h) return;
    free_all(h);
    delete h;
}

extern "C" const char* parrep_last_error(parrep_t h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" int parrep_ssa(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end, uint64_t seed,
                          double* hist_out, int64_t len, int64_t* events_out, float* kernel_ms, void* stream) {
    parrep_regions reg;
    memset(&reg, 0, sizeof(reg));
    reg.n = 1;
    reg.b[0] = 0;
    std::string why;
    if (!check_network(net, &reg, why)) return fail(nullptr, PARREP_EINVAL, why);
    if (precision != PARREP_FP64 && precision != PARREP_FP32) return fail(nullptr, PARREP_EINVAL, "precision");
    if (n_traj < 1 || n_traj > (1ll << 31)) return fail(nullptr, PARREP_EINVAL, "n_traj");
    if (!(T_end >= 0.0) || !(T_end < kTEndLimit)) return fail(nullptr, PARREP_EINVAL, "T_end");
    NetDev nd;
    std::vector<double> pU, pV, gU, gV;
    build_net(net, &reg, nd, pU, pV, gU, gV);
    const int nbins = nd.nbins;
    if (hist_out && len != nbins) return fail(nullptr, PARREP_EINVAL, "len != n_bins");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> pUf(pU.size()), pVf(pV.size());
    for (size_t i = 0; i < pU.size(); ++i) pUf[i] = (float)pU[i];
    for (size_t i = 0; i < pV.size(); ++i) pVf[i] = (float)pV[i];
    double *dpU = nullptr, *dpV = nullptr, *dout = nullptr;
    float *dpUf = nullptr, *dpVf = nullptr;
    unsigned long long *dh = nullptr, *dev_ev = nullptr;
    int* dst = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = upload(&dpU, pU);
    if (e == cudaSuccess) e = upload(&dpV, pV);
    if (e == cudaSuccess) e = upload(&dpUf, pUf);
    if (e == cudaSuccess) e = upload(&dpVf, pVf);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dh, sizeof(unsigned long long) * nbins);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, sizeof(double) * nbins);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dev_ev, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&dst, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int status = 0;
    unsigned long long evh = 0;
    if (e == cudaSuccess) {
        nd.prodU_d = dpU;
        nd.prodV_d = dpV;
        nd.prodU_f = dpUf;
        nd.prodV_f = dpVf;
        e = cudaMemsetAsync(dh, 0, sizeof(unsigned long long) * nbins, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dev_ev, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
            e = launch_ssa(nd, precision, n_traj, net->x0[0], net->n_species > 1 ? net->x0[1] : 0,
                           (unsigned long long)llrint(T_end * kQScale), seed, dh, dev_ev, dst, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess && hist_out) e = launch_hist_normalise(dh, dh, nbins, 0.0, dout, nullptr, nullptr, st);
        if (e == cudaSuccess && hist_out)
            e = cudaMemcpyAsync(hist_out, dout, sizeof(double) * nbins, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&evh, dev_ev, sizeof(evh), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, dst, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && kernel_ms) cudaEventElapsedTime(kernel_ms, e0, e1);
    }
    void* ptrs[] = {dpU, dpV, dpUf, dpVf, dh, dout, dev_ev, dst};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(nullptr, PARREP_ECUDA, std::string("parrep_ssa: ") + cudaGetErrorString(e));
    if (events_out) *events_out = (int64_t)evh;
    if (status) return fail(nullptr, status, "parrep_ssa: a state left [0, hist_max]");
    return PARREP_OK;
}

extern "C" int parrep_ssa_trace(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end,
                                uint64_t seed, int64_t max_steps, int32_t* reactions, int32_t* states,
                                double* holding, int64_t* n_jumps, int32_t* x_final) {
    parrep_regions reg;
    memset(&reg, 0, sizeof(reg));
    reg.n = 1;
    std::string why;
    if (!check_network(net, &reg, why)) return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: " + why);
    if (precision != PARREP_FP64 && precision != PARREP_FP32)
        return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: precision");
    if (n_traj < 1 || n_traj > (1ll << 24) || max_steps < 1 || n_traj * max_steps > (1ll << 28))
        return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: need 1 <= n_traj, 1 <= max_steps, n_traj*max_steps <= 2^28");
    if (!(T_end >= 0.0) || !(T_end < kTEndLimit)) return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: T_end");
    if (!reactions || !states || !n_jumps || !x_final)
        return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: null output");
    if (net->x0_uniform_hi != 0) return fail(nullptr, PARREP_EINVAL, "parrep_ssa_trace: x0_uniform_hi must be 0");
    NetDev nd;
    std::vector<double> pU, pV, gU, gV;
    build_net(net, &reg, nd, pU, pV, gU, gV);
    std::vector<float> pUf(pU.size()), pVf(pV.size());
    for (size_t i = 0; i < pU.size(); ++i) pUf[i] = (float)pU[i];
    for (size_t i = 0; i < pV.size(); ++i) pVf[i] = (float)pV[i];
    const size_t n = (size_t)n_traj * (size_t)max_steps;
    double *dpU = nullptr, *dpV = nullptr;
    float *dpUf = nullptr, *dpVf = nullptr;
    int *dJ = nullptr, *dst = nullptr;
    int2 *dx = nullptr, *dxf = nullptr;
    unsigned long long* dq = nullptr;
    long long* dn = nullptr;
    cudaError_t e = upload(&dpU, pU);
    if (e == cudaSuccess) e = upload(&dpV, pV);
    if (e == cudaSuccess) e = upload(&dpUf, pUf);
    if (e == cudaSuccess) e = upload(&dpVf, pVf);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dJ, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dx, sizeof(int2) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dq, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dn, sizeof(long long) * n_traj);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dxf, sizeof(int2) * n_traj);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dst, sizeof(int));
    int status = 0;
    std::vector<unsigned long long> hq;
    if (e == cudaSuccess) {
        nd.prodU_d = dpU;
        nd.prodV_d = dpV;
        nd.prodU_f = dpUf;
        nd.prodV_f = dpVf;
        e = cudaMemset(dst, 0, sizeof(int));
        if (e == cudaSuccess)
            e = launch_ssa_trace(nd, precision, n_traj, net->x0[0], net->n_species > 1 ? net->x0[1] : 0,
                                 (unsigned long long)llrint(T_end * kQScale), seed, max_steps, dJ, dx, dq, dn, dxf,
                                 dst, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(reactions, dJ, sizeof(int) * n, cudaMemcpyDefault);
        if (e == cudaSuccess) e = cudaMemcpy(states, dx, sizeof(int2) * n, cudaMemcpyDefault);
        if (e == cudaSuccess) e = cudaMemcpy(n_jumps, dn, sizeof(long long) * n_traj, cudaMemcpyDefault);
        if (e == cudaSuccess) e = cudaMemcpy(x_final, dxf, sizeof(int2) * n_traj, cudaMemcpyDefault);
        if (e == cudaSuccess && holding) {
            hq.resize(n);
            e = cudaMemcpy(hq.data(), dq, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost);
        }
        if (e == cudaSuccess) e = cudaMemcpy(&status, dst, sizeof(int), cudaMemcpyDeviceToHost);
    }
    void* ptrs[] = {dpU, dpV, dpUf, dpVf, dJ, dx, dq, dn, dxf, dst};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (e != cudaSuccess) return fail(nullptr, PARREP_ECUDA, std::string("parrep_ssa_trace: ") + cudaGetErrorString(e));
    if (holding) {
        std::vector<double> ht(n);
        for (size_t i = 0; i < n; ++i) ht[i] = (double)hq[i] * kQInv;
        if (cudaMemcpy(holding, ht.data(), sizeof(double) * n, cudaMemcpyDefault) != cudaSuccess)
            return fail(nullptr, PARREP_ECUDA, "parrep_ssa_trace: copy of the holding times");
    }
    if (status) return fail(nullptr, status, "parrep_ssa_trace: a state left [0, hist_max]");
    return PARREP_OK;
}

extern "C" int parrep_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out) {
    if (!ctr || !key || !out || n < 0) return fail(nullptr, PARREP_EINVAL, "parrep_philox: bad arguments");
    if (n == 0) return PARREP_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc((void**)&dc, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dk, sizeof(uint32_t) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, sizeof(uint32_t) * 2 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(dc, dk, n, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    if (dc) cudaFree(dc);
    if (dk) cudaFree(dk);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, PARREP_ECUDA, std::string("parrep_philox: ") + cudaGetErrorString(e));
    return PARREP_OK;
}
