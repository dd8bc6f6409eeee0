// parrep_ssa_noalloc: the plain-SSA entry point for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework that
// owns the whole device memory pool and forbids side allocations, and
// latency-sensitive loops in which cudaMalloc/cudaFree would synchronise the
// device.  This entry point runs the same kernel as parrep_ssa but keeps all
// of its scratch (the fixed-point histogram, the jump counter, the status word
// and the toggle rate tables) in one file-scope device array instead of
// allocating it.  The caller still passes the output buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "parrep.h"
#include "parrep_internal.h"
#include "parrep_handle.h"

using namespace parrep;

namespace {

// Layout of the scratch array (all offsets multiples of 256 bytes):
//   [hist: kMaxBins x u64][events: u64][status: int][pad to 256]
//   [prodU_d: kMaxTab x f64][prodV_d: kMaxTab x f64][prodU_f: kMaxTab x f32][prodV_f: kMaxTab x f32]
constexpr size_t kMaxBins = PARREP_SSA_NOALLOC_MAX_BINS;
constexpr size_t kMaxTab = PARREP_SSA_NOALLOC_MAX_SPECIES_STATES;
constexpr size_t kOffHist = 0;
constexpr size_t kOffEvents = kOffHist + kMaxBins * 8;
constexpr size_t kOffStatus = kOffEvents + 8;
constexpr size_t kOffTabUd = kOffEvents + 256;
constexpr size_t kOffTabVd = kOffTabUd + kMaxTab * 8;
constexpr size_t kOffTabUf = kOffTabVd + kMaxTab * 8;
constexpr size_t kOffTabVf = kOffTabUf + kMaxTab * 4;
constexpr size_t kScratchBytes = kOffTabVf + kMaxTab * 4;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_ssa_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {nullptr};

// Host staging of the toggle tables, also static (guarded by g_tab_mu).
std::mutex g_tab_mu;
double g_hUd[kMaxTab], g_hVd[kMaxTab];
float g_hUf[kMaxTab], g_hVf[kMaxTab];

// Device address of g_ssa_scratch on the current device.  In host code the
// name g_ssa_scratch is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_of_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ssa_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = (unsigned char*)p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace

// Errors go through fail() like parrep_ssa's, so parrep_last_error(NULL)
// names the reason.
static int noalloc_fail(int code, const std::string& why) {
    return fail(nullptr, code, "parrep_ssa_noalloc: " + why);
}

extern "C" int parrep_ssa_noalloc(const parrep_network* net, int32_t precision, int64_t n_traj, double T_end,
                                  uint64_t seed, double* hist_out, int64_t len, int64_t* events_out,
                                  void* stream) {
    if (!net || !hist_out) return noalloc_fail(PARREP_EINVAL, "null network or output");
    // the same network checks as parrep_ssa (one region: the plain SSA has no
    // metastable sets); check_network allocates nothing
    parrep_regions reg;
    memset(&reg, 0, sizeof(reg));
    reg.n = 1;
    std::string why;
    if (!check_network(net, &reg, why)) return noalloc_fail(PARREP_EINVAL, why);
    if (net->kind != PARREP_SCHLOGL && net->kind != PARREP_TOGGLE)
        return noalloc_fail(PARREP_EINVAL, "only the Schloegl and toggle networks");
    if (net->x0_uniform_hi != 0) return noalloc_fail(PARREP_EINVAL, "x0_uniform_hi is not used by the plain SSA");
    const int nsp = net->n_species;
    // sizes beyond the fixed scratch are refused, never truncated
    const long long nb = (long long)(net->hist_max[0] + 1) * (net->hist_max[1] + 1);
    if (nb > (long long)kMaxBins) return noalloc_fail(PARREP_EINVAL, "more histogram bins than the fixed scratch holds");
    if ((size_t)net->hist_max[0] + 1 > kMaxTab || (size_t)net->hist_max[1] + 1 > kMaxTab)
        return noalloc_fail(PARREP_EINVAL, "more states per species than the fixed scratch holds");
    if (len != nb) return noalloc_fail(PARREP_EINVAL, "len != n_bins");
    if (precision != PARREP_FP64 && precision != PARREP_FP32) return noalloc_fail(PARREP_EINVAL, "precision");
    if (n_traj < 1 || n_traj > (1ll << 31)) return noalloc_fail(PARREP_EINVAL, "n_traj");
    if (!(T_end >= 0.0) || !(T_end < kTEndLimit)) return noalloc_fail(PARREP_EINVAL, "T_end");
    const int x0 = net->x0[0], x1 = nsp > 1 ? net->x0[1] : 0;

    unsigned char* base = nullptr;
    cudaError_t e = scratch_of_current_device(&base);
    if (e != cudaSuccess) return noalloc_fail(PARREP_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;

    NetDev nd;
    memset(&nd, 0, sizeof(nd));
    nd.kind = net->kind;
    nd.nsp = nsp;
    nd.hist_max0 = net->hist_max[0];
    nd.hist_max1 = net->hist_max[1];
    nd.ystride = net->hist_max[1] + 1;
    nd.nbins = (int)nb;
    nd.nreg = 0;
    if (nsp == 1) {
        for (int j = 0; j < 4; ++j) {
            nd.A[j] = net->c[j] * net->s[j];
            nd.Af[j] = (float)nd.A[j];
        }
    } else {
        // production-rate tables, the same expressions as parrep_create's
        std::lock_guard<std::mutex> lock(g_tab_mu);
        const size_t nU = (size_t)net->hist_max[1] + 1, nV = (size_t)net->hist_max[0] + 1;
        for (size_t v = 0; v < nU; ++v) {
            g_hUd[v] = net->c[0] / (1.0 + pow((double)v, net->c[1]));
            g_hUf[v] = (float)g_hUd[v];
        }
        for (size_t u = 0; u < nV; ++u) {
            g_hVd[u] = net->c[3] / (1.0 + pow((double)u, net->c[4]));
            g_hVf[u] = (float)g_hVd[u];
        }
        nd.dU = net->c[2];
        nd.dV = net->c[5];
        nd.dUf = (float)net->c[2];
        nd.dVf = (float)net->c[5];
        nd.prodU_d = (const double*)(base + kOffTabUd);
        nd.prodV_d = (const double*)(base + kOffTabVd);
        nd.prodU_f = (const float*)(base + kOffTabUf);
        nd.prodV_f = (const float*)(base + kOffTabVf);
        e = cudaMemcpyAsync(base + kOffTabUd, g_hUd, nU * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffTabVd, g_hVd, nV * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffTabUf, g_hUf, nU * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffTabVf, g_hVf, nV * 4, cudaMemcpyHostToDevice, st);
        // the host tables are reused by the next call: wait until they are copied
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return noalloc_fail(PARREP_ECUDA, cudaGetErrorString(e));
    }
    unsigned long long* hist = (unsigned long long*)(base + kOffHist);
    unsigned long long* events = (unsigned long long*)(base + kOffEvents);
    int* status = (int*)(base + kOffStatus);
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(hist, 0, (size_t)nb * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(events, 0, 256, st);
    if (e == cudaSuccess)
        e = launch_ssa(nd, precision, n_traj, x0, x1, (unsigned long long)llrint(T_end * kQScale), seed, hist, events,
                       status, st);
    // fixed point -> time units in place (each thread reads then writes its own bin)
    if (e == cudaSuccess) e = launch_hist_normalise(hist, hist, (int)nb, 0.0, (double*)hist, nullptr, nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist_out, hist, (size_t)nb * 8, cudaMemcpyDefault, st);
    unsigned long long ev = 0;
    int stat = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ev, events, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&stat, status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(PARREP_ECUDA, cudaGetErrorString(e));
    if (events_out) *events_out = (int64_t)ev;
    if (stat) return noalloc_fail(stat, "a state left [0, hist_max]");
    return PARREP_OK;
}
