// Host side of parrep_uq (include/parrep.h): the stationary uncertainty
// quantification of Sec. IV.B over independent completed runs.  Checks that
// the samples share a network shape and a window, gathers their device
// views, and runs the two UQ kernels (parrep_kernels.cu) on the first
// handle's stream.
#include <cuda_runtime.h>

#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "parrep.h"
#include "parrep_handle.h"
#include "parrep_internal.h"

using namespace parrep;

namespace {

// Device scratch of one call, freed on every return path.
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = (T*)q;
        return e;
    }
};

}  // namespace

#define UQ_CK(h, call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

extern "C" int parrep_uq(const parrep_t* handles, int32_t n, const double* f, int64_t len, const double* dirs,
                         int32_t n_dirs, double* dir_bounds, double* Y_out, parrep_uq_result* out) {
    if (!handles || n < 1 || !handles[0]) return PARREP_EINVAL;
    parrep_t h0 = handles[0];
    if (n < 2) return fail(h0, PARREP_EINVAL, "the IAF estimator needs at least two samples");
    if (!f || !out) return fail(h0, PARREP_EINVAL, "f and out are required");
    if (n_dirs < 0 || (n_dirs > 0 && (!dirs || !dir_bounds)))
        return fail(h0, PARREP_EINVAL, "n_dirs > 0 needs dirs and dir_bounds");
    std::set<parrep_t> seen;
    double window = 0.0;
    std::vector<UqSample> smp(n);
    for (int k = 0; k < n; ++k) {
        parrep_t h = handles[k];
        if (!h) return fail(h0, PARREP_EINVAL, "NULL handle in the sample list");
        if (!seen.insert(h).second) return fail(h0, PARREP_EINVAL, "the same handle appears twice");
        if (!h->has_run) return fail(h0, PARREP_ESTATE, "a sample has no completed run");
        if (h->net.kind != h0->net.kind || h->net.hist_max[0] != h0->net.hist_max[0] ||
            h->net.hist_max[1] != h0->net.hist_max[1])
            return fail(h0, PARREP_EINVAL, "samples differ in network kind or hist_max");
        const double w = h->stats.T_s - h->T_burn;
        if (!(w > 0.0)) return fail(h0, PARREP_EINVAL, "empty window [T_burn, T_end]");
        if (k == 0) window = w;
        else if (w != window) return fail(h0, PARREP_EINVAL, "samples differ in T_end - T_burn");
        smp[k].net = h->nd;
        smp[k].c = h->d_c;
        smp[k].hist = h->d_hist_post;
        smp[k].gradU_n = h->d_gradU_n;
        smp[k].gradV_n = h->d_gradV_n;
    }
    if (len != h0->nbins) return fail(h0, PARREP_EINVAL, "len != n_bins");
    const int L = h0->L;
    cudaStream_t st = (cudaStream_t)h0->opt.stream;
    // the handles' runs completed on their own streams: order after them
    for (int k = 0; k < n; ++k)
        if (handles[k]->opt.stream != h0->opt.stream) UQ_CK(h0, cudaStreamSynchronize((cudaStream_t)handles[k]->opt.stream));
    Scratch s;
    UqSample* d_smp;
    double *d_f, *d_Y, *d_Z, *d_dirs = nullptr, *d_db = nullptr;
    UqOut* d_out;
    UQ_CK(h0, s.alloc(&d_smp, n));
    UQ_CK(h0, s.alloc(&d_f, (size_t)len));
    UQ_CK(h0, s.alloc(&d_Y, n));
    UQ_CK(h0, s.alloc(&d_Z, (size_t)n * 64));
    UQ_CK(h0, s.alloc(&d_out, 1));
    if (n_dirs > 0) {
        UQ_CK(h0, s.alloc(&d_dirs, (size_t)n_dirs * L));
        UQ_CK(h0, s.alloc(&d_db, n_dirs));
        UQ_CK(h0, cudaMemcpyAsync(d_dirs, dirs, sizeof(double) * n_dirs * L, cudaMemcpyDefault, st));
    }
    UQ_CK(h0, cudaMemcpyAsync(d_smp, smp.data(), sizeof(UqSample) * n, cudaMemcpyHostToDevice, st));
    UQ_CK(h0, cudaMemcpyAsync(d_f, f, sizeof(double) * len, cudaMemcpyDefault, st));
    UQ_CK(h0, launch_uq(d_smp, n, L, d_f, window, d_dirs, n_dirs, d_Y, d_Z, d_out, d_db, st));
    UqOut r;
    UQ_CK(h0, cudaMemcpyAsync(&r, d_out, sizeof(UqOut), cudaMemcpyDeviceToHost, st));
    if (Y_out) UQ_CK(h0, cudaMemcpyAsync(Y_out, d_Y, sizeof(double) * n, cudaMemcpyDefault, st));
    if (n_dirs > 0) UQ_CK(h0, cudaMemcpyAsync(dir_bounds, d_db, sizeof(double) * n_dirs, cudaMemcpyDefault, st));
    UQ_CK(h0, cudaStreamSynchronize(st));
    memset(out, 0, sizeof(*out));
    out->n_samples = n;
    out->n_params = L;
    out->window = window;
    out->iaf = r.iaf;
    out->mean_f = r.mean_f;
    for (int i = 0; i < L * L; ++i) {
        out->fim[i] = r.fim[i];
        out->fim_half_width[i] = r.half[i];
    }
    for (int j = 0; j < L; ++j) out->bound[j] = r.bound[j];
    return PARREP_OK;
}
