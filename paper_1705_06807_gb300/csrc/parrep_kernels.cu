// CUDA kernels of the ParRep library (sm_103a).
//
// One persistent cooperative launch runs Algorithm 1 of Wang & Plechac
// (arXiv 1705.06807, Sec. III.A) to T_end:
//   * decorrelation: one leader thread simulates X~ (serial by definition);
//   * dephasing: one thread per replica, lockstep jumps of the embedded chain,
//     Fleming-Viot respawn inside groups of <= 32 lanes by warp ballot and
//     shuffle (no memory traffic);
//   * parallel step: one thread per replica with its integer state in
//     registers runs S lockstep steps ahead ("a chunk"), stopping at its own
//     escape; a warp/block/grid minimum over the packed key (step, replica)
//     gives the paper's (N*, K).  Contributions tau and f(X) tau go straight
//     into a block-private shared-memory histogram in 64-bit fixed point.
//     A chunk that holds the escape, the T_end cut or the T_burn split is
//     rolled back and replayed exactly (the counter-based generator makes a
//     replay bit-identical), keeping only the contributions at or before the
//     cut in the paper's (step, replica) order.
// Every wait on another block is bounded by a no-progress timeout and turns
// into PARREP_ETIMEOUT instead of a hang.
//
// The file is compiled once per part (-DPARREP_PART=0..11) so that the
// persistent kernels, each of which inlines the whole of Algorithm 1, build
// in parallel: part 0 holds the small kernels and the dispatchers, parts 1-9
// instantiate the run, batch and serve kernels in each form (binary64,
// binary32 staged, binary32 direct), parts 10-11 the batch and serve kernels
// in the mixed binary32 form.
#include <cuda_runtime.h>
#include <stdint.h>

#include "parrep_internal.h"

#ifndef PARREP_PART
#define PARREP_PART 0
#endif

namespace parrep {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplies with the Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        unsigned hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        unsigned hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// uniform in (0,1): 52 bits, (m + 1/2) 2^-52 (exact in binary64)
__device__ __forceinline__ double u01d(unsigned a, unsigned b) {
    unsigned long long m = ((unsigned long long)a << 20) | (unsigned long long)(b >> 12);
    return ((double)m + 0.5) * 0x1p-52;
}
// uniform in (0,1): 23 bits, (m + 1/2) 2^-23 (exact in binary32)
__device__ __forceinline__ float u01f(unsigned w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

// uniform integer in {0..n-1}
__device__ __forceinline__ unsigned pick(unsigned w, unsigned n) { return __umulhi(w, n); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase timer of a block: thread 0 adds clock64 deltas per phase.
struct PhaseClock {
    unsigned long long acc[12];
    long long t;
    __device__ __forceinline__ void start() {
        if (threadIdx.x == 0) t = clock64();
    }
    __device__ __forceinline__ void lap(int phase) {
        if (threadIdx.x == 0) {
            const long long n = clock64();
            acc[phase] += (unsigned long long)(n - t);
            t = n;
        }
    }
};
enum { kPhDecorr = 0, kPhDephase = 1, kPhDraw = 2, kPhChain = 3, kPhAccount = 4, kPhBarrier = 5, kPhSpecial = 6,
       kPhVote = 7, kPhDecDraw = 8, kPhDecChain = 9, kPhDecTimes = 10, kPhDecCommit = 11 };

template <typename T>
__device__ __forceinline__ T ldv(const T* p) {
    return *(const volatile T*)p;
}

// Loads and stores that order against memory the host writes or reads
// (host-mapped rings and flags of the serving path).
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_sys(const int* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(int* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// network: propensities, selection, update, regions
// ---------------------------------------------------------------------------
__device__ __forceinline__ int region_of(const NetDev& N, int x0, int x1) {
    for (int i = 0; i < N.nreg; ++i) {
        long long v = (long long)N.ra0[i] * x0 + (long long)N.ra1[i] * x1;
        if (v < N.rb[i]) return i;
    }
    return N.nreg;
}

__device__ __forceinline__ bool out_of_range(const NetDev& N, int x0, int x1) {
    return x0 < 0 || x0 > N.hist_max0 || x1 < 0 || x1 > N.hist_max1;
}

// eta_J: Schloegl (+1,-1,+1,-1) on x0; toggle (+U,+V,-U,-V); genetic switch
// (x0 = 2m + xi, x1 = p): m+1, m-1, p+1, p-1, xi 0->1, xi 1->0
__device__ __forceinline__ void apply(const NetDev& N, int J, int& x0, int& x1) {
    if (N.kind == PARREP_SCHLOGL) {
        x0 += (J & 1) ? -1 : 1;
    } else if (N.kind == PARREP_GENETIC) {
        const int d = (J & 1) ? -1 : 1;
        if (J < 2) x0 += 2 * d;
        else if (J < 4) x1 += d;
        else x0 += d;
    } else {
        int d = (J < 2) ? 1 : -1;
        if (J & 1) x1 += d; else x0 += d;
    }
}

template <typename F>
__device__ __forceinline__ int select4(F l0, F l1, F l2, F l3, F target) {
    F cum = l0;
    if (cum > target) return 0;
    cum = cum + l1;
    if (cum > target) return 1;
    cum = cum + l2;
    if (cum > target) return 2;
    cum = cum + l3;
    if (cum > target) return 3;
    // rounding left no channel above the target: take the last positive one
    return l3 > (F)0 ? 3 : (l2 > (F)0 ? 2 : (l1 > (F)0 ? 1 : 0));
}

__device__ __forceinline__ void props_d(const NetDev& N, int x0, int x1, double& l0, double& l1, double& l2,
                                        double& l3) {
    if (N.kind == PARREP_SCHLOGL) {
        double xd = (double)x0;
        double h1 = xd * (xd - 1.0);
        double h2 = h1 * (xd - 2.0);
        l0 = N.A[0] * h1;
        l1 = N.A[1] * h2;
        l2 = N.A[2];
        l3 = N.A[3] * xd;
    } else {
        l0 = __ldg(N.prodU_d + x1);
        l1 = __ldg(N.prodV_d + x0);
        l2 = N.dU * (double)x0;
        l3 = N.dV * (double)x1;
    }
}

// The genetic switch in binary64 (Sec. V.B, Table IV): the six propensities
// from x0 = 2m + xi, x1 = p, with F(p), G(p) from the host-built tables.
__device__ __forceinline__ void props6_d(const NetDev& N, int x0, int x1, double l[6]) {
    const double xi = (double)(x0 & 1), m = (double)(x0 >> 1);
    l[0] = N.A[0] * xi;
    l[1] = N.A[1] * m;
    l[2] = N.A[2] * m;
    l[3] = (double)x1;
    l[4] = __ldg(N.prodU_d + x1) * (1.0 - xi);
    l[5] = __ldg(N.prodV_d + x1) * xi;
}

// Total rate a0 in binary64, summed left to right over the network's channels.
__device__ __forceinline__ double a0_d(const NetDev& N, int x0, int x1) {
    if (N.kind == PARREP_GENETIC) {
        double l[6];
        props6_d(N, x0, x1, l);
        return ((((l[0] + l[1]) + l[2]) + l[3]) + l[4]) + l[5];
    }
    double l0, l1, l2, l3;
    props_d(N, x0, x1, l0, l1, l2, l3);
    return ((l0 + l1) + l2) + l3;
}

__device__ __forceinline__ void props_f(const NetDev& N, int x0, int x1, float& l0, float& l1, float& l2,
                                        float& l3) {
    if (N.kind == PARREP_SCHLOGL) {
        float xf = (float)x0;
        float h1 = xf * (xf - 1.0f);
        float h2 = h1 * (xf - 2.0f);
        l0 = N.Af[0] * h1;
        l1 = N.Af[1] * h2;
        l2 = N.Af[2];
        l3 = N.Af[3] * xf;
    } else {
        l0 = __ldg(N.prodU_f + x1);
        l1 = __ldg(N.prodV_f + x0);
        l2 = N.dUf * (float)x0;
        l3 = N.dVf * (float)x1;
    }
}

// round(tau * 2^40) of a finite binary32 tau >= 0 by integer operations on its
// bits (half-way cases round up), saturated at 2^62 -- no 64-bit conversion
// instruction, which GB300 would issue on its narrow FP64 pipe.
__device__ __forceinline__ unsigned long long q_of_f32(float tau) {
    const unsigned b = __float_as_uint(tau);
    const int be = (int)(b >> 23);
    if (be == 0) return 0ull;  // zero or subnormal
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
    const int e = be - 110;  // tau * 2^40 = m * 2^(be - 127 - 23 + 40)
    if (e >= 0) return e > 38 ? (1ull << 62) : (m << e);
    if (e < -25) return 0ull;
    return (m + (1ull << (-e - 1))) >> (-e);
}

// One Gillespie direct-method step at (x0,x1) from the Philox words w:
// returns J and (if WANT_TAU) the holding time tau = -log(u1)/a0 in fixed point.
// Words of parallel step n of replica r, and of decorrelation step `step`.
// The FP32 form needs two 23-bit uniforms per step, so one Philox call serves
// the step pair (2p, 2p+1): words 0,1 for the even step, 2,3 for the odd one.
template <bool F32>
__device__ __forceinline__ uint4 par_words(unsigned r, unsigned n, unsigned cycle, uint2 key) {
    if (!F32) return philox10(make_uint4(r, n, cycle, kTagParallel), key);
    const uint4 w = philox10(make_uint4(r, n >> 1, cycle, kTagParallel), key);
    return (n & 1) ? make_uint4(w.z, w.w, 0u, 0u) : w;
}
template <bool F32>
__device__ __forceinline__ uint4 decorr_words(unsigned long long step, unsigned cycle, uint2 key) {
    const unsigned long long c = F32 ? step >> 1 : step;
    const uint4 w = philox10(make_uint4((unsigned)(c >> 32), (unsigned)c, cycle, kTagDecorr), key);
    return (F32 && (step & 1)) ? make_uint4(w.z, w.w, 0u, 0u) : w;
}

// FP32 form: w.x and w.y are the step's two words (a Philox call serves two
// steps: words 0,1 for the even and 2,3 for the odd step).
template <bool F32, bool WANT_TAU>
__device__ __forceinline__ int ssa_draw(const NetDev& N, int x0, int x1, uint4 w, unsigned long long& q) {
    if (F32 && N.kind == PARREP_GENETIC) {
        // six channels in binary32: F(p), G(p) from the binary32 tables
        const float xi = (float)(x0 & 1), m = (float)(x0 >> 1);
        float l[6];
        l[0] = N.Af[0] * xi;
        l[1] = N.Af[1] * m;
        l[2] = N.Af[2] * m;
        l[3] = (float)x1;
        l[4] = __ldg(N.prodU_f + x1) * (1.0f - xi);
        l[5] = __ldg(N.prodV_f + x1) * xi;
        const float a0 = ((((l[0] + l[1]) + l[2]) + l[3]) + l[4]) + l[5];
        if (WANT_TAU) q = q_of_f32(-logf(u01f(w.x)) * __frcp_rn(a0));
        const float t = u01f(w.y) * a0;
        float cum = l[0];
        if (cum > t) return 0;
#pragma unroll
        for (int j = 1; j < 6; ++j) {
            cum = cum + l[j];
            if (cum > t) return j;
        }
        int J = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (l[j] > 0.0f) J = j;
        return J;
    } else if (F32) {
        float l0, l1, l2, l3;
        props_f(N, x0, x1, l0, l1, l2, l3);
        float a0 = ((l0 + l1) + l2) + l3;
        if (WANT_TAU) q = q_of_f32(-logf(u01f(w.x)) * __frcp_rn(a0));
        return select4<float>(l0, l1, l2, l3, u01f(w.y) * a0);
    } else if (N.kind == PARREP_GENETIC) {
        double l[6];
        props6_d(N, x0, x1, l);
        const double a0 = ((((l[0] + l[1]) + l[2]) + l[3]) + l[4]) + l[5];
        if (WANT_TAU) {
            const double tau = -log(u01d(w.x, w.y)) / a0;
            q = __double2ull_rn(tau * 0x1p40);
            if (q > (1ull << 62)) q = 1ull << 62;
        }
        // direct method over six channels, sums left to right; if rounding
        // leaves no sum above the target, the last channel with lambda > 0
        const double t = u01d(w.z, w.w) * a0;
        double cum = l[0];
        if (cum > t) return 0;
#pragma unroll
        for (int j = 1; j < 6; ++j) {
            cum = cum + l[j];
            if (cum > t) return j;
        }
        int J = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (l[j] > 0.0) J = j;
        return J;
    } else {
        double l0, l1, l2, l3;
        props_d(N, x0, x1, l0, l1, l2, l3);
        double a0 = ((l0 + l1) + l2) + l3;
        if (WANT_TAU) {
            const double tau = -log(u01d(w.x, w.y)) / a0;
            q = __double2ull_rn(tau * 0x1p40);
            if (q > (1ull << 62)) q = 1ull << 62;
        }
        return select4<double>(l0, l1, l2, l3, u01d(w.z, w.w) * a0);
    }
}

__device__ __forceinline__ uint2 seed_key(unsigned long long seed) {
    return make_uint2((unsigned)seed, (unsigned)(seed >> 32));
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_min(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

struct BlockScratch {
    unsigned long long a[32], b[32], c[32], d[32];
};

// Block reduction of (min a, min b, sum c, sum d); thread 0 gets the result.
__device__ __forceinline__ void block_reduce4(BlockScratch& s, unsigned long long& a, unsigned long long& b,
                                              unsigned long long& c, unsigned long long& d) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_min(a);
    b = warp_min(b);
    c = warp_sum(c);
    d = warp_sum(d);
    if (lane == 0) {
        s.a[wid] = a;
        s.b[wid] = b;
        s.c[wid] = c;
        s.d[wid] = d;
    }
    __syncthreads();
    if (wid == 0) {
        a = lane < nw ? s.a[lane] : kNone;
        b = lane < nw ? s.b[lane] : kNone;
        c = lane < nw ? s.c[lane] : 0ull;
        d = lane < nw ? s.d[lane] : 0ull;
        a = warp_min(a);
        b = warp_min(b);
        c = warp_sum(c);
        d = warp_sum(d);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// grid barrier, bounded: a wait that sees no progress for timeout_ns sets
// PARREP_ETIMEOUT and returns; every caller leaves the kernel on a nonzero
// status.  The barrier counts calls so that a test can make block 0 skip one.
// ---------------------------------------------------------------------------
// Longest sleep between polls of a waiting block (one thread per block
// polls): short, so that a barrier releases within a fraction of a microsecond.
#ifndef PARREP_BARRIER_SLEEP_MAX_NS
#define PARREP_BARRIER_SLEEP_MAX_NS 128
#endif
constexpr unsigned kBarrierSleepMaxNs = PARREP_BARRIER_SLEEP_MAX_NS;

struct BarState {
    int index;
    int lb, nblk;  // this block's index among the blocks serving the instance, and their number
};

static __device__ bool grid_sync(const RunParams& P, BarState& bs) {
    __shared__ int ok;
    RunCtl* ctl = P.ctl;
    const int idx = bs.index++;
    // lanes that skipped a leader-only stretch wait for it here: a block
    // barrier needs the whole warp at the same instruction
    __syncwarp();
    __syncthreads();
    if (P.stall_barrier >= 0 && idx == P.stall_barrier && bs.lb == 0) {
        // fault injection: block 0 leaves without arriving
        return false;
    }
    if (threadIdx.x == 0) {
        const unsigned g = ldv(&ctl->bar_gen);
        __threadfence();
        atomicAdd(P.progress, 1ull);
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == (unsigned)bs.nblk - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            unsigned long long t0 = globaltimer();
            unsigned long long p0 = ldv(P.progress);
            unsigned ns = 32;
            while (ldv(&ctl->bar_gen) == g) {
                if (ldv(&ctl->status) != 0) break;
                __nanosleep(ns);
                if (ns < kBarrierSleepMaxNs) ns <<= 1;
                const unsigned long long p = ldv(P.progress);
                const unsigned long long t = globaltimer();
                if (p != p0) {
                    p0 = p;
                    t0 = t;
                } else if ((long long)(t - t0) > P.timeout_ns) {
                    atomicCAS(&ctl->status, 0, PARREP_ETIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        // one read per block, so that every thread of the block takes the same branch
        ok = ldv(&ctl->status) == 0;
    }
    __syncwarp();
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------------------
// leader (block 0, thread 0): initial state and decorrelation
// ---------------------------------------------------------------------------
static __device__ void leader_contribute(const RunParams& P, RunCtl* ctl, int x0, int x1, unsigned long long q,
                                  unsigned long long& Ts, int& burn_done, bool& ended,
                                  unsigned long long* sh = nullptr, int sh_post = 0) {
    const NetDev& N = P.net;
    unsigned long long t = q;
    const unsigned long long rem = P.q_Tend - Ts;
    if (t >= rem) {
        t = rem;
        ended = true;
    }
    unsigned long long pre = 0, post = t;
    if (!burn_done) {
        const unsigned long long room = P.q_Tburn - Ts;
        pre = t < room ? t : room;
        post = t - pre;
        if (t >= room) burn_done = 1;
    }
    const int bin = x0 * N.ystride + x1;
    // block 0's shared histogram feeds the period sh_post says (the leader is
    // its only writer during the decorrelation); else the global sums
    if (pre) {
        if (sh && !sh_post) sh[bin] += pre;
        else atomicAdd(P.hist_pre + bin, pre);
    }
    if (post) {
        if (sh && sh_post) sh[bin] += post;
        else atomicAdd(P.hist_post + bin, post);
    }
    Ts += t;
}

static __device__ void leader_log(const RunParams& P, RunCtl* ctl, const CycleRecDev& rec) {
    long long i = ctl->log_n;
    if (i < P.log_cap) P.log[i] = rec;
    ctl->log_n = i + 1;
}

// End of a decorrelation (leader): n_p of the coming dephasing, the cycle
// record's first half, the shared state for the other blocks.
static __device__ void leader_finish_decorr(const RunParams& P, int x0, int x1, int W, unsigned long long Ts, int burn_done,
                                     unsigned long long step, bool ended, int status, unsigned cycle) {
    RunCtl* ctl = P.ctl;
    const NetDev& N = P.net;
    ctl->ev_decorr += step;
    long long np = 0;
    if (!ended && status == 0) {
        if (P.thresh == PARREP_THRESH_STEPS) {
            np = P.n_p;
        } else {
            const double a0 = a0_d(N, x0, x1);
            const double n = ceil(P.t_phase * a0);
            if (!(n < 4294967295.0)) status = PARREP_ERANGE;
            else np = (long long)n;
        }
    }
    ctl->xt0 = x0;
    ctl->xt1 = x1;
    ctl->W = W;
    ctl->Ts = Ts;
    ctl->burn_done = burn_done;
    ctl->np = np;
    // the cycle record is completed when the cycle ends; keep its first part
    CycleRecDev rec;
    rec.cycle = cycle;
    rec.W = W;
    rec.ended = ended ? 1 : 0;
    rec.decorr_steps = (long long)step;
    rec.dephase_steps = np;
    rec.n_star = 0;
    rec.k = -1;
    rec.xt0 = x0;
    rec.xt1 = x1;
    rec.Ts = Ts;
    if (ended || status) {
        if (ended) leader_log(P, ctl, rec);
        ctl->cycles += 1;
        ctl->done = 1;
    } else {
        // stash for the end of the cycle
        if (ctl->log_n < P.log_cap) P.log[ctl->log_n] = rec;
    }
    if (status) atomicCAS(&ctl->status, 0, status);
    __threadfence();
}


template <bool F32>
static __device__ void leader_decorrelate(const RunParams& P) {
    RunCtl* ctl = P.ctl;
    const NetDev& N = P.net;
    const uint2 key = seed_key(P.seed);
    int x0 = ctl->xt0, x1 = ctl->xt1;
    unsigned long long Ts = ctl->Ts;
    int burn_done = ctl->burn_done;
    const unsigned cycle = ctl->cycle;
    int W = region_of(N, x0, x1);
    long long Nc = 0;
    unsigned long long inW = 0;
    unsigned long long step = 0;
    bool ended = false;
    int status = 0;
    for (;;) {
        if (P.thresh == PARREP_THRESH_STEPS ? (Nc >= P.n_c) : (inW >= P.q_tcorr)) break;
        const uint4 w = decorr_words<F32>(step, cycle, key);
        unsigned long long q = 0;
        const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
        ++step;
        leader_contribute(P, ctl, x0, x1, q, Ts, burn_done, ended);
        if (ended) break;
        apply(N, J, x0, x1);
        if (out_of_range(N, x0, x1)) {
            status = PARREP_ERANGE;
            break;
        }
        const int Wn = region_of(N, x0, x1);
        if (Wn == W) {
            ++Nc;
            inW += q;
        } else {
            Nc = 0;
            inW = 0;
            W = Wn;
        }
        if ((step & 4095ull) == 0) atomicAdd(&ctl->progress, 1ull);
    }
    leader_finish_decorr(P, x0, x1, W, Ts, burn_done, step, ended, status, cycle);
}

// ---------------------------------------------------------------------------
// dephasing (Algorithm 1): n_p lockstep jumps of the embedded chain; after
// each, replicas that left W copy a uniformly chosen survivor of their group
// (fv_group consecutive lanes of the warp), or X~ if the group has none.
// All lanes of the warp execute the loop (inactive lanes carry no replica).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int kth_set_bit(unsigned m, unsigned k) {
    for (unsigned i = 0; i < k; ++i) m &= m - 1;
    return __ffs(m) - 1;
}

template <bool F32>
static __device__ int dephase_warp(const NetDev& N, bool active, unsigned r, int G, int W, int xt0, int xt1, long long np,
                            unsigned cycle, uint2 key, int& x0, int& x1) {
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, active);
    x0 = xt0;
    x1 = xt1;
    if (act == 0) return 0;
    const unsigned gm = (G >= 32) ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
    for (long long i = 0; i < np; ++i) {
        int n0 = x0, n1 = x1;
        bool ex = false, bad = false;
        if (active) {
            uint4 w;
            if (F32) {  // one Philox call per four jumps, word i mod 4
                if ((i & 3) == 0) w4 = philox10(make_uint4(r, (unsigned)(i >> 2), cycle, kTagDephase), key);
                const unsigned wi = (i & 3) == 0 ? w4.x : (i & 3) == 1 ? w4.y : (i & 3) == 2 ? w4.z : w4.w;
                w = make_uint4(0u, wi, 0u, 0u);
            } else {
                w = philox10(make_uint4(r, (unsigned)i, cycle, kTagDephase), key);
            }
            unsigned long long q;
            const int J = ssa_draw<F32, false>(N, x0, x1, w, q);
            apply(N, J, n0, n1);
            ex = region_of(N, n0, n1) != W;
            bad = !ex && out_of_range(N, n0, n1);
        }
        const unsigned exm = __ballot_sync(0xffffffffu, ex);
        if (__ballot_sync(0xffffffffu, bad)) return PARREP_ERANGE;
        if (exm) {
            const unsigned sm = act & ~exm & gm;
            int src = lane;
            if (ex) {
                const int ns = __popc(sm);
                if (ns > 0) {
                    uint4 w = philox10(make_uint4(r, (unsigned)i, cycle, kTagFV), key);
                    src = kth_set_bit(sm, pick(w.x, (unsigned)ns));
                } else {
                    src = -1;
                }
            }
            const int s0 = __shfl_sync(0xffffffffu, n0, src < 0 ? lane : src);
            const int s1 = __shfl_sync(0xffffffffu, n1, src < 0 ? lane : src);
            if (ex) {
                n0 = src < 0 ? xt0 : s0;
                n1 = src < 0 ? xt1 : s1;
            }
        }
        x0 = n0;
        x1 = n1;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// parallel step helpers
// ---------------------------------------------------------------------------
// Where a block's holding times go.  GB300 has no native 64-bit shared-memory
// atomic add (it is emulated and serialises under contention), so the FP32
// form splits q into two 32-bit limbs -- the low 16 bits and the rest -- added
// with native 32-bit atomics and folded exactly into the 64-bit shared sums
// every fold_period(B, RB) staged sub-chunks (at most).  A sub-chunk adds at most
// B*RB values to a bin, so with q < qmax = 2^47 / (B*RB*fold_period) the
// high-limb sum stays inside a signed 32-bit range (roll-backs included) and
// the low-limb sum below 2^30.  Holding times too large for the limbs go
// straight to the global sums.
struct HistSink {
    unsigned long long* sh;  // shared histogram or nullptr
    unsigned long long* g;   // global histogram of the current period
    unsigned* lo;            // FP32 form: limbs of the shared histogram
    unsigned* hi;
    int ystride;
    unsigned long long qmax;
    __device__ __forceinline__ void add(int x0, int x1, unsigned long long q) const {
        const int b = x0 * ystride + x1;
        if (lo && q < qmax) {
            atomicAdd(lo + b, (unsigned)(q & 0xffffu));
            atomicAdd(hi + b, (unsigned)(q >> 16));
        } else if (sh && !lo) {
            atomicAdd(sh + b, q);
        } else {
            atomicAdd(g + b, q);
        }
    }
    __device__ __forceinline__ void sub(int x0, int x1, unsigned long long q) const {
        const int b = x0 * ystride + x1;
        if (lo && q < qmax) {
            atomicAdd(lo + b, 0u - (unsigned)(q & 0xffffu));
            atomicAdd(hi + b, 0u - (unsigned)(q >> 16));
        } else if (sh && !lo) {
            atomicAdd(sh + b, 0ull - q);
        } else {
            atomicAdd(g + b, 0ull - q);
        }
    }
};

// Sub-chunks between limb folds in the pipelined parallel step: as many as
// keep B * RB * period at 4096 (qmax = 2^35), at least one.
__device__ __forceinline__ int fold_period(int B, int log2RB) {
    const int n = 4096 / (B << log2RB);
    return n > 1 ? n : 1;
}

// Folds the limbs of bins [b0, b1] into the 64-bit shared sums (signed, so a
// roll-back's negative limb sums are exact) and clears them.
__device__ __forceinline__ void fold_limbs(const HistSink& hs, int b0, int b1, int ystride, int c0, int c1,
                                           int tid = -1, int T = 0) {
    if (tid < 0) {
        tid = threadIdx.x;
        T = blockDim.x;
    }
    // bins of the rectangle rows [b0, b1] x columns [c0, c1]
    const int w = c1 - c0 + 1;
    const int n = (b1 - b0 + 1) * w;
    for (int k = tid; k < n; k += T) {
        const int row = b0 + k / w, col = c0 + k % w;
        const int b = row * ystride + col;
        const int vl = (int)hs.lo[b], vh = (int)hs.hi[b];
        if (vl | vh) {
            hs.sh[b] += (unsigned long long)(((long long)vh << 16) + (long long)vl);
            hs.lo[b] = 0;
            hs.hi[b] = 0;
        }
    }
}

__device__ __forceinline__ unsigned long long pos_of(int s, unsigned r) {
    return ((unsigned long long)(unsigned)s << 32) | (unsigned long long)r;
}

enum ReplayMode { kRollback = 0, kStepSum = 1, kTauAt = 2, kPrecise = 3 };

struct Cuts {
    unsigned long long posC;  // replica contributions after this are never included
    unsigned long long posE;  // escape cut (N*, K), in-chunk
    unsigned long long posT, partT;
    unsigned long long posB, partB;
    int nB, nT;               // steps of the T_burn / T_end crossing (-1: none)
};

// Re-simulates the chunk of replica r from (x0,x1) exactly as the first pass.
template <bool F32, int MODE>
static __device__ void replay_chunk(const RunParams& P, const HistSink& hs, int x0, int x1, unsigned r, int W,
                             unsigned cycle, unsigned n0, int S, const Cuts& cut, bool to_post,
                             unsigned long long& inc_q, unsigned long long& inc_ev, unsigned long long& ev) {
    const NetDev& N = P.net;
    const uint2 key = seed_key(P.seed);
    uint4 wp = make_uint4(0u, 0u, 0u, 0u);
    for (int s = 0; s < S; ++s) {
        const unsigned long long pos = pos_of(s, r);
        if (MODE != kRollback && pos > cut.posC) break;
        const unsigned n = n0 + (unsigned)s;
        uint4 w;
        if (F32) {  // one Philox call per step pair (n0 is even)
            if ((n & 1u) == 0u) wp = philox10(make_uint4(r, n >> 1, cycle, kTagParallel), key);
            w = (n & 1u) ? make_uint4(wp.z, wp.w, 0u, 0u) : wp;
        } else {
            w = par_words<F32>(r, n, cycle, key);
        }
        unsigned long long q = 0;
        const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
        ++ev;
        if (MODE == kRollback) {
            hs.sub(x0, x1, q);
        } else if (MODE == kStepSum) {
            atomicAdd(P.step_sum + s, q);
        } else if (MODE == kTauAt) {
            if (s == cut.nB) P.tau_at[r] = q;
            if (s == cut.nT) P.tau_at[P.R + r] = q;
        } else {
            if (pos > cut.posE || pos > cut.posT) break;
            unsigned long long amt = (pos == cut.posT) ? cut.partT : q;
            // the T_burn split: before the cut to the global pre-burn sums,
            // after it to the (post-burn) sink
            unsigned long long pre = 0, post = amt;
            if (cut.posB != kNone) {
                if (pos < cut.posB) {
                    pre = amt;
                    post = 0;
                } else if (pos == cut.posB) {
                    pre = cut.partB < amt ? cut.partB : amt;
                    post = amt - pre;
                }
            }
            const int b = x0 * P.net.ystride + x1;
            if (pre) atomicAdd(P.hist_pre + b, pre);
            if (post) {
                if (hs.sh) atomicAdd(hs.sh + b, post);
                else atomicAdd((to_post ? P.hist_post : P.hist_pre) + b, post);
            }
            inc_q += amt;
            if (pos == cut.posT) break;  // the run ends inside this holding time
            inc_ev += 1;
        }
        int n0_ = x0, n1_ = x1;
        apply(N, J, n0_, n1_);
        if (out_of_range(N, n0_, n1_)) break;
        if (region_of(N, n0_, n1_) != W) break;
        x0 = n0_;
        x1 = n1_;
    }
}

// The step-sum pass of replay_chunk for a whole warp: every lane walks the
// chunk in step with the others (a replica that escaped, left the range or
// passed the cut adds zero), the warp sums each step's holding times with
// shuffles and one lane adds the sum to step_sum[s] -- one global atomic per
// warp and step instead of one per replica (thousands of replicas would
// otherwise queue on the same address).  The sums are exact integers, so the
// result is the same.
template <bool F32>
static __device__ void replay_stepsum_warp(const RunParams& P, bool active, int x0, int x1, unsigned r, int W,
                                           unsigned cycle, unsigned n0, int S, const Cuts& cut,
                                           unsigned long long& ev) {
    const NetDev& N = P.net;
    const uint2 key = seed_key(P.seed);
    const int lane = threadIdx.x & 31;
    bool live = active;
    uint4 wp = make_uint4(0u, 0u, 0u, 0u);
    for (int s = 0; s < S; ++s) {
        unsigned long long q = 0;
        if (live) {
            if (pos_of(s, r) > cut.posC) {
                live = false;
            } else {
                const unsigned n = n0 + (unsigned)s;
                uint4 w;
                if (F32) {  // one Philox call per step pair (n0 is even)
                    if ((n & 1u) == 0u) wp = philox10(make_uint4(r, n >> 1, cycle, kTagParallel), key);
                    w = (n & 1u) ? make_uint4(wp.z, wp.w, 0u, 0u) : wp;
                } else {
                    w = par_words<F32>(r, n, cycle, key);
                }
                const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
                ++ev;
                int a0 = x0, a1 = x1;
                apply(N, J, a0, a1);
                if (out_of_range(N, a0, a1) || region_of(N, a0, a1) != W) {
                    live = false;
                } else {
                    x0 = a0;
                    x1 = a1;
                }
            }
        }
        unsigned long long v = q;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(P.step_sum + s, v);
        if (!__any_sync(0xffffffffu, live)) break;
    }
}

static __device__ void flush_shared(unsigned long long* sh, unsigned long long* g, int nbins) {
    __syncwarp();
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const unsigned long long v = sh[b];
        if (v) atomicAdd(g + b, v);
        sh[b] = 0;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// FP32 form: staged chunks.  Per sub-chunk of B steps, three phases: (P) the
// helper threads draw Philox words for the block's replicas -- independent
// work with no dependency chain; (C) the replica owners advance their states
// through the B steps, reading the uniforms (for the Schloegl network, their
// 23-bit indices, compared with a per-state threshold table) from shared
// memory, and write the pre-jump states to a trace; (A) the helpers turn the
// trace into holding times and accumulate them.  An owner's serial chain is
// thus only the choice of the reaction and the update.  In the pipelined
// layout the phases of consecutive sub-chunks overlap (chunk_f32).
// ---------------------------------------------------------------------------
struct FastSmem {
    const float* inv;    // Schloegl: per state RN(1/a0) (nullptr: none)
    const int4* thr;     // Schloegl: per state choice thresholds (choice_thresholds; nullptr: none)
    int* rng;            // [4]: min/max of x0 and x1 touched in the sub-chunk
    unsigned long long* decp;  // decorrelation rounds: prefix sums of the holding times
    const float* prodU;  // toggle: production of U by V, of V by U (shared copies)
    const float* prodV;
    float2* buf;         // [B][RB]: (E = -log u1, u2), or (E, k2) for the threshold chain
    int* trace;          // [B][RB]: pre-jump state
    int* live;           // [RB]: replica still running in this chunk
    int* nvalid;         // [RB]: steps of the replica in this sub-chunk
};

template <int KIND>
__device__ __forceinline__ float4 cums_f32(const NetDev& N, const FastSmem& F, int x0, int x1) {
    if (KIND == PARREP_SCHLOGL) {
        float l0, l1, l2, l3;
        props_f(N, x0, 0, l0, l1, l2, l3);
        const float c1 = l0 + l1, c2 = c1 + l2;
        return make_float4(l0, c1, c2, c2 + l3);
    }
    const float l0 = F.prodU[x1], l1 = F.prodV[x0];
    const float l2 = N.dUf * (float)x0, l3 = N.dVf * (float)x1;
    const float c1 = l0 + l1, c2 = c1 + l2;
    return make_float4(l0, c1, c2, c2 + l3);
}

// The direct-method choice from the cumulative sums: the number of sums <= t
// is the first j with sum_j > t (the sums are non-decreasing).
template <int KIND>
__device__ __forceinline__ int pick_channel(const NetDev& N, float4 c, float u2, int x0, int x1) {
    const float t = u2 * c.w;
    int J = (int)(c.x <= t) + (int)(c.y <= t) + (int)(c.z <= t) + (int)(c.w <= t);
    if (J == 4) {  // rounding left no channel above the target
        float l0, l1, l2, l3;
        props_f(N, x0, x1, l0, l1, l2, l3);
        J = l3 > 0.f ? 3 : (l2 > 0.f ? 2 : (l1 > 0.f ? 1 : 0));
    }
    return J;
}

__device__ __forceinline__ int pack_state(int nsp, int x0, int x1) { return nsp > 1 ? (x0 | (x1 << 16)) : x0; }
__device__ __forceinline__ void unpack_state(int nsp, int p, int& x0, int& x1) {
    x0 = nsp > 1 ? (p & 0xffff) : p;
    x1 = nsp > 1 ? (p >> 16) : 0;
}

static __device__ void build_fast_tables(const NetDev& N, float* inv, float* pU, float* pV) {
    if (N.kind == PARREP_SCHLOGL) {
        // per state RN(1/a0)
        if (inv)
            for (int x = threadIdx.x; x <= N.hist_max0; x += blockDim.x) {
                float l0, l1, l2, l3;
                props_f(N, x, 0, l0, l1, l2, l3);
                const float c1 = l0 + l1, c2 = c1 + l2;
                inv[x] = __frcp_rn(c2 + l3);
            }
    } else {
        for (int v = threadIdx.x; v <= N.hist_max1; v += blockDim.x) pU[v] = N.prodU_f[v];
        for (int u = threadIdx.x; u <= N.hist_max0; u += blockDim.x) pV[u] = N.prodV_f[u];
    }
}

// (P) Philox words for steps step0 .. step0+nsteps-1 of the block's live replicas.
// The parallel step stores (E, u2) per step, or (E, k2) -- the 23-bit index
// of u2, as integer bits -- for the Schloegl threshold chain (F.thr).
template <bool WANT_E>
__device__ __forceinline__ void produce_store(const FastSmem& F, int lg, int mask, int nsteps, int i, uint4 w) {
    constexpr int PER = WANT_E ? 2 : 4;
    const int lane = i & mask, s = (i >> lg) * PER;
    if (!F.live[lane]) return;
    float2* buf = F.buf;
    if (WANT_E) {
        const bool kidx = F.thr != nullptr;
        const float ya = kidx ? __int_as_float((int)(w.y >> 9)) : u01f(w.y);
        const float yb = kidx ? __int_as_float((int)(w.w >> 9)) : u01f(w.w);
        buf[(s << lg) + lane] = make_float2(-logf(u01f(w.x)), ya);
        if (s + 1 < nsteps) buf[((s + 1) << lg) + lane] = make_float2(-logf(u01f(w.z)), yb);
    } else {
        buf[(s << lg) + lane].y = u01f(w.x);
        if (s + 1 < nsteps) buf[((s + 1) << lg) + lane].y = u01f(w.y);
        if (s + 2 < nsteps) buf[((s + 2) << lg) + lane].y = u01f(w.z);
        if (s + 3 < nsteps) buf[((s + 3) << lg) + lane].y = u01f(w.w);
    }
}

template <bool WANT_E>
__device__ __forceinline__ void produce_lanes(const RunParams& P, const FastSmem& F, unsigned rbase, unsigned step0,
                                              int nsteps, unsigned cycle, unsigned tag, uint2 key,
                                              int tid = -1, int T = 0) {
    // A Philox call serves PER consecutive steps of one replica: two in the
    // parallel step (u1, u2 each), four in the dephasing (u2 only).  step0 is
    // a multiple of PER.  Item i is (lane i % RB, call i / RB); T and the item
    // count are multiples of 32, so whether an item exists is warp-uniform and
    // no thread computes a call that is not needed.
    if (tid < 0) {
        tid = threadIdx.x;
        T = blockDim.x;
    }
    constexpr int PER = WANT_E ? 2 : 4;
    const int lg = P.log2RB, mask = P.RB - 1;
    const int total = ((nsteps + PER - 1) / PER) << lg;
    const unsigned g0 = step0 / PER;
    int i = tid;
    // two independent calls per pass while both exist, so that their rounds interleave
    for (; i + T < total; i += 2 * T) {
        const int j = i + T;
        const uint4 wa = philox10(make_uint4(rbase + (unsigned)(i & mask), g0 + (unsigned)(i >> lg), cycle, tag), key);
        const uint4 wb = philox10(make_uint4(rbase + (unsigned)(j & mask), g0 + (unsigned)(j >> lg), cycle, tag), key);
        produce_store<WANT_E>(F, lg, mask, nsteps, i, wa);
        produce_store<WANT_E>(F, lg, mask, nsteps, j, wb);
    }
    if (i < total) {
        const uint4 wa = philox10(make_uint4(rbase + (unsigned)(i & mask), g0 + (unsigned)(i >> lg), cycle, tag), key);
        produce_store<WANT_E>(F, lg, mask, nsteps, i, wa);
    }
}

// Region test of the owners' chains.  One species: W is the interval
// [lo, hi]; a state outside it left W or left [0, hist_max], which the rare
// branch tells apart.  Two species: the half-plane tests with coefficients
// held in registers.
struct RegionTest {
    int lo, hi;           // one species: the interval of W
    int n;                // number of half-plane tests
    int a0[4], a1[4];
    long long b[4];
    int ilo[5], ihi[5];   // one species: all region intervals
    int W;
    // all loads with constant indices: a runtime index into the kernel
    // parameters would turn into a slow generic load
    __device__ __forceinline__ void load(const NetDev& N) {
        n = N.nreg;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a0[i] = N.ra0[i];
            a1[i] = N.ra1[i];
            b[i] = N.rb[i];
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ilo[i] = N.wlo[i];
            ihi[i] = N.whi[i];
        }
    }
    __device__ __forceinline__ void set(int W_) {
        W = W_;
        lo = 1;
        hi = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (i == W_) {
                lo = ilo[i];
                hi = ihi[i];
            }
    }
    __device__ __forceinline__ void init(const NetDev& N, int W_) {
        load(N);
        set(W_);
    }
    // region of a one-species state inside [0, hist_max]
    __device__ __forceinline__ int region1(int x) const {
        int r = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (x >= ilo[i] && x <= ihi[i]) r = i;
        return r;
    }
    __device__ __forceinline__ int region2(int x0, int x1) const {
        int r = n;
#pragma unroll
        for (int i = 3; i >= 0; --i)
            if (i < n && (long long)a0[i] * x0 + (long long)a1[i] * x1 < b[i]) r = i;
        return r;
    }
    __device__ __forceinline__ int region(int nsp, int x0, int x1) const {
        return nsp == 1 ? region1(x0) : region2(x0, x1);
    }
};

// Outcome of a jump to (a0, a1): 0 = stays in W, 1 = escape, 2 = outside
// [0, hist_max].  In the parallel step and the decorrelation a jump outside
// the range is an error even if it also leaves W (OOB_FIRST); in the
// dephasing a replica that left W is replaced, whatever its state.
template <int KIND, bool OOB_FIRST>
__device__ __forceinline__ int jump_outcome(const NetDev& N, const RegionTest& rt, int a0, int a1) {
    if (KIND == PARREP_SCHLOGL) {
        if (a0 >= rt.lo && a0 <= rt.hi) return 0;
        const bool oob = a0 < 0 || a0 > N.hist_max0;
        if (OOB_FIRST) return oob ? 2 : 1;
        return oob ? (region_of(N, a0, 0) != rt.W ? 1 : 2) : 1;
    }
    if (OOB_FIRST && out_of_range(N, a0, a1)) return 2;
    if (rt.region2(a0, a1) != rt.W) return 1;
    return out_of_range(N, a0, a1) ? 2 : 0;
}

__device__ __forceinline__ int count_le(float4 c, float t) {
    return (int)(c.x <= t) + (int)(c.y <= t) + (int)(c.z <= t) + (int)(c.w <= t);
}

// J == 4: rounding left no cumulative sum above the target; the direct
// method then takes the last channel with positive propensity.
static __device__ __noinline__ int last_positive(const NetDev& N, int x0, int x1) {
    float l0, l1, l2, l3;
    props_f(N, x0, x1, l0, l1, l2, l3);
    return l3 > 0.f ? 3 : (l2 > 0.f ? 2 : (l1 > 0.f ? 1 : 0));
}

// Cumulative propensities of the Schloegl network at x in binary32, the same
// operations as props_f (so the same bits as the oracle's binary32 mode).
__device__ __forceinline__ float4 cums_schlogl(float A0, float A1, float A2, float A3, int x) {
    const float xf = (float)x;
    const float h1 = xf * (xf - 1.0f);
    const float h2 = h1 * (xf - 2.0f);
    const float l0 = A0 * h1, l1 = A1 * h2, l3 = A3 * xf;
    const float c1 = l0 + l1, c2 = c1 + A2;
    return make_float4(l0, c1, c2, c2 + l3);
}

__device__ __forceinline__ bool goes_up(float4 C, float t) { return (t < C.x) | ((C.y <= t) & (t < C.z)); }

// Speculative pass of a Schloegl jump chain over n steps (n even) from x, two
// steps per iteration, with no branch: the propensities at x-1, x, x+1 are
// computed together, the direct-method choice of a +-1 chain is "up" iff
// t < c0 or c1 <= t < c2, and the state is kept inside [lo, hi] so that it
// stays a valid table index.  trace[s*stride + off] receives the state before
// step s.  Returns the first step whose choice needed the rounding rule or
// whose target left [lo, hi] (n if none): every state up to and including
// that step's pre-jump state is exact.
__device__ __forceinline__ int spec_pass_schlogl(const NetDev& N, const float2* buf, int* trace, int stride, int off,
                                                 int n, int lo, int hi, int& x, int& mn, int& mx, int s0 = 0) {
    const float A0 = N.Af[0], A1 = N.Af[1], A2 = N.Af[2], A3 = N.Af[3];
    int first = n;
    const int npair = s0 + ((n - s0) & ~1);
    for (int s = s0; s < npair; s += 2) {
        const int i1 = s * stride + off, i2 = i1 + stride;
        const float ua = buf[i1].y, ub = buf[i2].y;
        const float4 C = cums_schlogl(A0, A1, A2, A3, x);
        const float4 L = cums_schlogl(A0, A1, A2, A3, x - 1);
        const float4 R = cums_schlogl(A0, A1, A2, A3, x + 1);
        const float t1 = ua * C.w, tR = ub * R.w, tL = ub * L.w;
        const bool up1 = goes_up(C, t1);
        const int xa = up1 ? x + 1 : x - 1;
        const bool up2 = up1 ? goes_up(R, tR) : goes_up(L, tL);
        const int xb = up2 ? xa + 1 : xa - 1;
        const bool r1 = (t1 >= C.w) | (xa < lo) | (xa > hi);
        const bool r2 = ((up1 ? tR : tL) >= (up1 ? R.w : L.w)) | (xb < lo) | (xb > hi);
        first = min(first, r1 ? s : (r2 ? s + 1 : n));
        trace[i1] = x;
        trace[i2] = xa;
        mn = min(mn, min(x, xa));
        mx = max(mx, max(x, xa));
        x = min(max(xb, lo), hi);
    }
    if (npair < n) {  // odd tail: one step
        const int i = npair * stride + off;
        const float4 C = cums_schlogl(A0, A1, A2, A3, x);
        const float t = buf[i].y * C.w;
        const int xa = goes_up(C, t) ? x + 1 : x - 1;
        first = min(first, ((t >= C.w) | (xa < lo) | (xa > hi)) ? npair : n);
        trace[i] = x;
        mn = min(mn, x);
        mx = max(mx, x);
        x = min(max(xa, lo), hi);
    }
    return first;
}

// Choice thresholds of the binary32 direct method at a Schloegl state.  A
// step's uniform is u_k = (k + 1/2) 2^-23 with k its 23-bit index, and the
// target t = RN(u_k a0) does not decrease with k; so "t >= c_j" holds exactly
// for k >= K_j, with K_j found by bisection on k (the same products and
// comparisons as the chain's).  The chain goes up (channels 0 and 2) iff
// k < K0 or K1 <= k < K2.  When rounding leaves no sum above t (k >= K3) the
// direct method takes the last channel with positive propensity, which goes
// up only if l3 = 0; then a0 = c2 exactly, K3 = K2, and the up set is k < K0
// or k >= K1.  Stored as (K0, K1, D): up iff k < K0 or (unsigned)(k - K1) < D.
static __device__ unsigned first_k_at_least(float a0, float c) {
    unsigned lo = 0u, hi = 1u << 23;  // the answer lies in [lo, hi]
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        const float u = ((float)mid + 0.5f) * 0x1p-23f;
        if (u * a0 >= c) hi = mid;
        else lo = mid + 1u;
    }
    return lo;
}

static __device__ int4 choice_thresholds(const NetDev& N, int x) {
    const float4 C = cums_schlogl(N.Af[0], N.Af[1], N.Af[2], N.Af[3], x);
    const unsigned K0 = first_k_at_least(C.w, C.x), K1 = first_k_at_least(C.w, C.y);
    const unsigned K2 = first_k_at_least(C.w, C.z);
    const bool rounding_up = (last_positive(N, x, 0) & 1) == 0;
    return make_int4((int)K0, (int)K1, (int)(rounding_up ? (1u << 23) - K1 : K2 - K1), 0);
}

__device__ __forceinline__ bool goes_up_k(int4 T, int k) {
    return (k < T.x) | ((unsigned)(k - T.y) < (unsigned)T.z);
}

// thr[x] for x in [-kThrPad, hist_max + kThrPad]; the entries beyond
// [0, hist_max] repeat the end states' (read only by speculative steps past an exit)
static __device__ void build_thr_table(const NetDev& N, int4* thr) {
    for (int k = threadIdx.x; k <= N.hist_max0 + 2 * kThrPad; k += blockDim.x)
        thr[k - kThrPad] = choice_thresholds(N, min(max(k - kThrPad, 0), N.hist_max0));
}

// Shared-memory accesses by shared-window address.  The staged arrays are
// reached through pointers kept in a struct, which the compiler may turn into
// generic accesses; the owner's chain reads and writes shared memory directly.
// The table reads are plain (the table does not change while a chain runs);
// the buffer reads and trace writes keep their order against the barriers.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int4 lds_table(unsigned a) {
    int4 v;
    asm("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ int lds_word(unsigned a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_word(unsigned a, int v) {
    asm volatile("st.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Speculative pass of a Schloegl jump chain with the threshold table: two
// steps per iteration, the entries at x-1, x, x+1 loaded together, and every
// choice exact.  trace[s*stride + off] receives the state before step s.
// Returns the first step whose target leaves [lo, hi] (n if none); the walk
// goes on past it (at most n steps, inside the table's padding) but nothing
// after that step is used.
__device__ __forceinline__ int spec_pass_thr(const int4* __restrict__ thr, const float2* buf, int* trace, int stride,
                                             int off, int n, int lo, int hi, int& x) {
    int first = n;
    const unsigned span = (unsigned)(hi - lo);
    const int npair = n & ~1;
    // .y of buf[i] (the 23-bit index) at ka + 8 i; thr[x] at ta + 16 x; trace[i] at ra + 4 i
    const unsigned ka = smem_addr(buf) + 4u, ta = smem_addr(thr), ra = smem_addr(trace);
    for (int s = 0; s < npair; s += 2) {
        const int i1 = s * stride + off, i2 = i1 + stride;
        const int k1 = lds_word(ka + 8u * (unsigned)i1), k2 = lds_word(ka + 8u * (unsigned)i2);
        const unsigned tx = ta + 16u * (unsigned)x;
        const int4 T0 = lds_table(tx), Tm = lds_table(tx - 16u), Tp = lds_table(tx + 16u);
        const bool up1 = goes_up_k(T0, k1);
        const bool up2 = up1 ? goes_up_k(Tp, k2) : goes_up_k(Tm, k2);
        const int xa = up1 ? x + 1 : x - 1;
        const int xb = up2 ? xa + 1 : xa - 1;
        const bool e1 = (unsigned)(xa - lo) > span, e2 = (unsigned)(xb - lo) > span;
        first = min(first, e1 ? s : (e2 ? s + 1 : n));
        sts_word(ra + 4u * (unsigned)i1, x);
        sts_word(ra + 4u * (unsigned)i2, xa);
        x = xb;
    }
    if (npair < n) {  // odd tail: one step
        const int i = npair * stride + off;
        const int xa = goes_up_k(thr[x], __float_as_int(buf[i].y)) ? x + 1 : x - 1;
        first = min(first, (unsigned)(xa - lo) > span ? npair : n);
        trace[i] = x;
        x = xa;
    }
    return first;
}

// (C) one owner's B lockstep steps of the parallel step; stops at its escape
// or at a state outside [0, hist_max].  Schloegl with its table: two steps
// per iteration -- the sums at x-1, x, x+1 are loaded together and the second
// choice is made for both outcomes of the first.
template <int KIND>
__device__ __forceinline__ void consume_par(const RunParams& P, const FastSmem& F, const RegionTest& rt,
                                            bool& running, int& x0, int& x1, unsigned r, int sbase,
                                            unsigned long long& mykey, unsigned long long& myoob, int& xe0,
                                            int& xe1) {
    const NetDev& N = P.net;
    const int lane = threadIdx.x;
    int nv = 0;
    int lo0 = 0x7fffffff, hi0 = -1, lo1 = 0x7fffffff, hi1 = -1;
    if (running) {
        nv = P.B;
        if (KIND == PARREP_SCHLOGL && F.thr) {
            // speculative pass with exact choices; the states it visits lie
            // within B of the start, which bounds the warp's rectangle
            const int B = P.B, lg = P.log2RB;
            int x = x0;
            lo0 = max(x0 - B, 0);
            hi0 = min(x0 + B, N.hist_max0);
            const int first = spec_pass_thr(F.thr, F.buf, F.trace, P.RB, lane, B, rt.lo, rt.hi, x);
            if (first < B) {
                // the replica leaves W (or [0, hist_max]) at step `first`
                const int i = (first << lg) + lane;
                const int y = F.trace[i];
                const int yn = goes_up_k(F.thr[y], __float_as_int(F.buf[i].y)) ? y + 1 : y - 1;
                if (jump_outcome<KIND, true>(N, rt, yn, 0) == 1) {
                    mykey = pos_of(sbase + first, r);
                    xe0 = yn;
                    xe1 = 0;
                } else {
                    myoob = pos_of(sbase + first, r);
                }
                nv = first + 1;
                running = false;
                x = y;
            }
            x0 = x;
        } else if (KIND == PARREP_SCHLOGL) {
            // speculative pass, then the exact rule from the first rare step on
            const int B = P.B, lg = P.log2RB;
            int x = x0;
            const int first = spec_pass_schlogl(N, F.buf, F.trace, P.RB, lane, B, rt.lo, rt.hi, x, lo0, hi0);
            if (first < B) {
                int y = F.trace[(first << lg) + lane];
                for (int s = first; s < B; ++s) {
                    const int i = (s << lg) + lane;
                    F.trace[i] = y;
                    lo0 = min(lo0, y);
                    hi0 = max(hi0, y);
                    const float4 c = cums_schlogl(N.Af[0], N.Af[1], N.Af[2], N.Af[3], y);
                    int J = count_le(c, F.buf[i].y * c.w);
                    if (J == 4) J = last_positive(N, y, 0);
                    const int yn = y + ((J & 1) ? -1 : 1);
                    const int o = jump_outcome<KIND, true>(N, rt, yn, 0);
                    if (o) {
                        if (o == 1) {
                            mykey = pos_of(sbase + s, r);
                            xe0 = yn;
                            xe1 = 0;
                        } else {
                            myoob = pos_of(sbase + s, r);
                        }
                        nv = s + 1;
                        running = false;
                        break;
                    }
                    y = yn;
                }
                x = y;
            }
            x0 = x;
        } else {
            for (int s = 0; s < P.B; ++s) {
                const int i = (s << P.log2RB) + lane;
                const float4 c = cums_f32<KIND>(N, F, x0, x1);
                int J = count_le(c, F.buf[i].y * c.w);
                if (J == 4) J = last_positive(N, x0, x1);
                F.trace[i] = pack_state(N.nsp, x0, x1);
                lo0 = min(lo0, x0);
                hi0 = max(hi0, x0);
                lo1 = min(lo1, x1);
                hi1 = max(hi1, x1);
                int a0 = x0, a1 = x1;
                apply(N, J, a0, a1);
                const int o = jump_outcome<KIND, true>(N, rt, a0, a1);
                if (o) {
                    if (o == 1) {
                        mykey = pos_of(sbase + s, r);
                        xe0 = a0;
                        xe1 = a1;
                    } else {
                        myoob = pos_of(sbase + s, r);
                    }
                    nv = s + 1;
                    running = false;
                    break;
                }
                x0 = a0;
                x1 = a1;
            }
        }
        if (!running) F.live[lane] = 0;
    }
    F.nvalid[lane] = nv;
    // the rectangle of states this warp touched, for folding the limbs
    if (KIND == PARREP_SCHLOGL) {
        lo1 = 0;
        hi1 = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo0 = min(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
        hi0 = max(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
        lo1 = min(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
        hi1 = max(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    }
    if ((lane & 31) == 0 && hi0 >= 0) {
        atomicMin(F.rng + 0, lo0);
        atomicMax(F.rng + 1, hi0);
        atomicMin(F.rng + 2, lo1);
        atomicMax(F.rng + 3, hi1);
    }
}

enum ChunkMode { kFirst = 4 };

// (A) the holding times of the sub-chunk's trace, used as the mode says:
// first pass (add), roll-back (subtract), per-step sums, one step's
// per-replica values, or the precise pass that keeps what precedes the cut.
// Accounts for K items base, base + T, ... (all of which exist).
template <int KIND, int MODE, int K>
__device__ __forceinline__ void account_items(const RunParams& P, const FastSmem& F, const HistSink& hs,
                                              unsigned rbase, int sbase, const Cuts& cut, bool to_post,
                                              unsigned long long& qs, unsigned long long& ev,
                                              unsigned long long& ev2, int base, int T, bool tabbed) {
    const NetDev& N = P.net;
    const int lg = P.log2RB, mask = P.RB - 1;
    int xa[K], xb[K];
    unsigned long long qv[K];
    bool ok[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int i = base + k * T;
        const int lane = i & mask, s = i >> lg;
        ok[k] = s < F.nvalid[lane];
        unpack_state(N.nsp, ok[k] ? F.trace[i] : 0, xa[k], xb[k]);
        const float ia0 = tabbed ? F.inv[xa[k]] : __frcp_rn(cums_f32<KIND>(N, F, xa[k], xb[k]).w);
        qv[k] = q_of_f32(F.buf[i].x * ia0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!ok[k]) continue;
        const int i = base + k * T;
        const int lane = i & mask, s = i >> lg;
        const int x0 = xa[k], x1 = xb[k];
        const unsigned long long q = qv[k];
        const int sc = sbase + s;
        const unsigned rr = rbase + (unsigned)lane;
        if (MODE == kFirst) {
            hs.add(x0, x1, q);
            qs += q;
            ++ev;
        } else if (MODE == kRollback) {
            hs.sub(x0, x1, q);
            ++ev;
        } else {
            const unsigned long long pos = pos_of(sc, rr);
            if (pos > cut.posC) continue;
            ++ev;
            if (MODE == kStepSum) {
                atomicAdd(P.step_sum + sc, q);
            } else if (MODE == kTauAt) {
                if (sc == cut.nB) P.tau_at[rr] = q;
                if (sc == cut.nT) P.tau_at[P.R + rr] = q;
            } else {
                if (pos > cut.posE || pos > cut.posT) continue;
                const unsigned long long amt = (pos == cut.posT) ? cut.partT : q;
                unsigned long long pre = 0, post = amt;
                if (cut.posB != kNone) {
                    if (pos < cut.posB) {
                        pre = amt;
                        post = 0;
                    } else if (pos == cut.posB) {
                        pre = cut.partB < amt ? cut.partB : amt;
                        post = amt - pre;
                    }
                }
                const int b = x0 * N.ystride + x1;
                if (pre) atomicAdd(P.hist_pre + b, pre);
                if (post) {
                    if (hs.sh) hs.add(x0, x1, post);
                    else atomicAdd((to_post ? P.hist_post : P.hist_pre) + b, post);
                }
                qs += amt;                   // included time
                if (pos != cut.posT) ++ev2;  // included jumps (the truncated one does not jump)
            }
        }
    }
}

template <int KIND, int MODE>
__device__ __forceinline__ void account(const RunParams& P, const FastSmem& F, const HistSink& hs, unsigned rbase,
                                        int sbase, const Cuts& cut, bool to_post, unsigned long long& qs,
                                        unsigned long long& ev, unsigned long long& ev2, int tid = -1, int T = 0) {
    if (tid < 0) {
        tid = threadIdx.x;
        T = blockDim.x;
    }
    const int total = P.B << P.log2RB;
    const bool tabbed = KIND == PARREP_SCHLOGL && F.inv;
    // Items i = step * RB + lane.  T and total are multiples of 32, so the
    // bounds below are warp-uniform: up to four items per pass while four
    // exist (their loads and conversions interleave), then one at a time.
    int base = tid;
    for (; base + 3 * T < total; base += 4 * T)
        account_items<KIND, MODE, 4>(P, F, hs, rbase, sbase, cut, to_post, qs, ev, ev2, base, T, tabbed);
    if (base + T < total) {
        account_items<KIND, MODE, 2>(P, F, hs, rbase, sbase, cut, to_post, qs, ev, ev2, base, T, tabbed);
        base += 2 * T;
    }
    if (base < total) account_items<KIND, MODE, 1>(P, F, hs, rbase, sbase, cut, to_post, qs, ev, ev2, base, T, tabbed);
}

// One chunk (S steps) of the parallel step for the whole block, in a mode.
// Every thread of the block calls it; owners carry the replica states.
template <int KIND, int MODE>
static __device__ void chunk_f32(const RunParams& P, const FastSmem& F, const HistSink& hs, bool active, unsigned rbase,
                          unsigned r, const RegionTest& rt, unsigned cycle, unsigned n0, int S, uint2 key, int& x0,
                          int& x1, const Cuts& cut, bool to_post, unsigned long long& mykey, unsigned long long& myoob,
                          int& xe0, int& xe1, unsigned long long& qs, unsigned long long& ev,
                          unsigned long long& inc_ev, PhaseClock& pc) {
    const bool owner = threadIdx.x < P.RB;
    bool running = owner && active;
    const bool limbs = hs.lo != nullptr && MODE != kStepSum && MODE != kTauAt;
    if (P.pipelined) {
        // Warp-specialised pipeline: in stage j the owner warps walk
        // sub-chunk j while the helper warps draw sub-chunk j+1 and account
        // for sub-chunk j-1 (draws in three slots, traces in two), so the
        // owners' serial chains overlap the helpers' parallel work.  One
        // block barrier per stage; every fold_period sub-chunks (and at the
        // end) the helpers fold the limbs of the states the owners touched
        // since the last fold, behind a named barrier of their own.
        const int RB = P.RB, B = P.B;
        const int nh = blockDim.x - RB, h = threadIdx.x - RB;
        const int slotsz = B << P.log2RB;
        const int fp = fold_period(P.B, P.log2RB);
        if (owner) F.live[threadIdx.x] = running ? 1 : 0;
        // two per-sub-chunk rectangles of touched states and their union since the last fold
        if (threadIdx.x < 12) F.rng[threadIdx.x] = (threadIdx.x & 1) ? -1 : 0x7fffffff;
        __syncthreads();
        pc.start();
        const int nsub = S / B;
        if (!owner) {
            FastSmem Fp = F;
            produce_lanes<true>(P, Fp, rbase, n0, B, cycle, kTagParallel, key, h, nh);
        }
        __syncthreads();
        pc.lap(kPhDraw);
        bool any = true;
        for (int j = 0;; ++j) {
            const bool consume = any && j < nsub;
            if (owner) {
                if (consume) {
                    FastSmem Fj = F;
                    Fj.buf = F.buf + (j % 3) * slotsz;
                    Fj.trace = F.trace + (j & 1) * slotsz;
                    Fj.nvalid = F.nvalid + (j & 1) * RB;
                    Fj.rng = F.rng + (j & 1) * 4;
                    consume_par<KIND>(P, Fj, rt, running, x0, x1, r, j * B, mykey, myoob, xe0, xe1);
                } else {
                    F.nvalid[(j & 1) * RB + threadIdx.x] = 0;
                }
            } else {
                if (consume && j + 1 < nsub) {
                    FastSmem Fp = F;
                    Fp.buf = F.buf + ((j + 1) % 3) * slotsz;
                    produce_lanes<true>(P, Fp, rbase, n0 + (unsigned)((j + 1) * B), B, cycle, kTagParallel, key,
                                        h, nh);
                }
                if (j >= 1) {
                    const int jp = j - 1;
                    FastSmem Fa = F;
                    Fa.buf = F.buf + (jp % 3) * slotsz;
                    Fa.trace = F.trace + (jp & 1) * slotsz;
                    Fa.nvalid = F.nvalid + (jp & 1) * RB;
                    account<KIND, MODE>(P, Fa, hs, rbase, jp * B, cut, to_post, qs, ev, inc_ev, h, nh);
                    int* rg = F.rng + (jp & 1) * 4;
                    int* un = F.rng + 8;
                    if (h < 4) {
                        const int v = rg[h];
                        un[h] = (h & 1) ? max(un[h], v) : min(un[h], v);
                        rg[h] = (h & 1) ? -1 : 0x7fffffff;
                    }
                    if (limbs && (!consume || jp % fp == fp - 1)) {
                        asm volatile("bar.sync 1, %0;" ::"r"(nh) : "memory");
                        if (un[1] >= un[0]) fold_limbs(hs, un[0], un[1], P.net.ystride, un[2], un[3], h, nh);
                        asm volatile("bar.sync 1, %0;" ::"r"(nh) : "memory");
                        if (h < 4) un[h] = (h & 1) ? -1 : 0x7fffffff;
                    }
                }
            }
            const bool any_next = __syncthreads_or(running);
            pc.lap(kPhChain);
            if (!consume) break;
            any = any_next;
        }
        return;
    }
    if (owner) F.live[threadIdx.x] = running ? 1 : 0;
    if (threadIdx.x == 0) {
        F.rng[0] = 0x7fffffff;
        F.rng[1] = -1;
        F.rng[2] = 0x7fffffff;
        F.rng[3] = -1;
    }
    __syncthreads();
    for (int sub = 0; sub < S; sub += P.B) {
        pc.start();
        produce_lanes<true>(P, F, rbase, n0 + (unsigned)sub, P.B, cycle, kTagParallel, key);
        __syncthreads();
        pc.lap(kPhDraw);
        if (owner) consume_par<KIND>(P, F, rt, running, x0, x1, r, sub, mykey, myoob, xe0, xe1);
        __syncthreads();
        pc.lap(kPhChain);
        account<KIND, MODE>(P, F, hs, rbase, sub, cut, to_post, qs, ev, inc_ev);
        const bool any = __syncthreads_or(running);
        if (limbs) {
            const int r0 = F.rng[0], r1 = F.rng[1], c0 = F.rng[2], c1 = F.rng[3];
            if (r1 >= r0) fold_limbs(hs, r0, r1, P.net.ystride, c0, c1);
            __syncthreads();
            if (threadIdx.x == 0) {
                F.rng[0] = 0x7fffffff;
                F.rng[1] = -1;
                F.rng[2] = 0x7fffffff;
                F.rng[3] = -1;
            }
            __syncthreads();
        }
        pc.lap(kPhAccount);
        if (!any) break;
    }
}

// Dephasing of the FP32 form: the uniforms of B lockstep jumps at a time come
// from shared memory; the owner warps run the jumps and the Fleming-Viot
// ballots exactly as dephase_warp does.
template <int KIND>
static __device__ int dephase_f32(const RunParams& P, const FastSmem& F, const RegionTest& rt, bool active, unsigned rbase,
                           unsigned r, int xt0, int xt1, long long np, unsigned cycle, uint2 key, int& x0, int& x1) {
    const NetDev& N = P.net;
    const bool owner = threadIdx.x < P.RB;  // whole warps, RB is a multiple of 32
    const int lane = threadIdx.x & 31;
    const int G = P.G;
    x0 = xt0;
    x1 = xt1;
    if (owner) F.live[threadIdx.x] = active ? 1 : 0;
    __syncthreads();
    unsigned act = 0, gm = 0;
    if (owner) {
        act = __ballot_sync(0xffffffffu, active);
        gm = (G >= 32) ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    }
    int err = 0;
    // pipelined layout: the helper warps draw batch k + 1 into the other draw
    // slot while the owner warps walk batch k (one block barrier a batch)
    const bool pipe = P.pipelined != 0;
    const int slotsz = P.B << P.log2RB;
    const int nh = (int)blockDim.x - P.RB, h = (int)threadIdx.x - P.RB;
    if (pipe) {
        if (!owner)
            produce_lanes<false>(P, F, rbase, 0u, (int)(np < (long long)P.B ? np : (long long)P.B), cycle, kTagDephase,
                                 key, h, nh);
        __syncthreads();
    }
    long long kb = 0;
    for (long long i0 = 0; i0 < np; i0 += P.B, ++kb) {
        const int nb = (int)((np - i0) < (long long)P.B ? (np - i0) : (long long)P.B);
        FastSmem Fb = F;
        if (pipe) {
            Fb.buf = F.buf + (int)(kb & 1) * slotsz;
            const long long i1 = i0 + P.B;
            if (!owner && i1 < np) {
                FastSmem Fn = F;
                Fn.buf = F.buf + (int)((kb + 1) & 1) * slotsz;
                produce_lanes<false>(P, Fn, rbase, (unsigned)i1, (int)((np - i1) < (long long)P.B ? (np - i1) : P.B),
                                     cycle, kTagDephase, key, h, nh);
            }
        } else {
            produce_lanes<false>(P, F, rbase, (unsigned)i0, nb, cycle, kTagDephase, key);
            __syncthreads();
        }
        if (owner && act && !err && KIND == PARREP_SCHLOGL) {
            // every lane speculates through the sub-chunk; the warp goes back
            // to the first step at which any lane met an escape or the
            // rounding rule, takes that step exactly (with Fleming-Viot), and
            // speculates again from the next one
            const int lg = P.log2RB;
            int sb = 0;
            while (sb < nb) {
                int x = x0, mn = 0, mx = 0;
                int first = spec_pass_schlogl(N, Fb.buf, F.trace, P.RB, threadIdx.x, nb, rt.lo, rt.hi, x, mn, mx, sb);
                if (!active) first = nb;
                int fw = first;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) fw = min(fw, __shfl_xor_sync(0xffffffffu, fw, o));
                if (fw == nb) {
                    if (active) x0 = x;
                    break;
                }
                if (active) x0 = F.trace[(fw << lg) + threadIdx.x];
                const unsigned i = (unsigned)i0 + (unsigned)fw;
                int n0 = x0, n1 = x1;
                bool ex = false, bad = false;
                if (active) {
                    const float4 c = cums_schlogl(N.Af[0], N.Af[1], N.Af[2], N.Af[3], x0);
                    int J = count_le(c, Fb.buf[(fw << lg) + threadIdx.x].y * c.w);
                    if (J == 4) J = last_positive(N, x0, x1);
                    apply(N, J, n0, n1);
                    const int o = jump_outcome<KIND, false>(N, rt, n0, n1);
                    ex = o == 1;
                    bad = o == 2;
                }
                const unsigned exm = __ballot_sync(0xffffffffu, ex);
                if (__ballot_sync(0xffffffffu, bad)) {
                    err = PARREP_ERANGE;
                    break;
                }
                if (exm) {
                    const unsigned sm = act & ~exm & gm;
                    int src = lane;
                    if (ex) {
                        const int ns = __popc(sm);
                        if (ns > 0) {
                            uint4 w = philox10(make_uint4(r, i, cycle, kTagFV), key);
                            src = kth_set_bit(sm, pick(w.x, (unsigned)ns));
                        } else {
                            src = -1;
                        }
                    }
                    const int s0 = __shfl_sync(0xffffffffu, n0, src < 0 ? lane : src);
                    const int s1 = __shfl_sync(0xffffffffu, n1, src < 0 ? lane : src);
                    if (ex) {
                        n0 = src < 0 ? xt0 : s0;
                        n1 = src < 0 ? xt1 : s1;
                    }
                }
                x0 = n0;
                x1 = n1;
                sb = fw + 1;
            }
        } else if (owner && act && !err) {
            for (int s = 0; s < nb; ++s) {
                const unsigned i = (unsigned)i0 + (unsigned)s;
                int n0 = x0, n1 = x1;
                bool ex = false, bad = false;
                if (active) {
                    const float4 c = cums_f32<KIND>(N, Fb, x0, x1);
                    int J = count_le(c, Fb.buf[(s << P.log2RB) + threadIdx.x].y * c.w);
                    if (J == 4) J = last_positive(N, x0, x1);
                    apply(N, J, n0, n1);
                    const int o = jump_outcome<KIND, false>(N, rt, n0, n1);
                    ex = o == 1;
                    bad = o == 2;
                }
                const unsigned exm = __ballot_sync(0xffffffffu, ex);
                if (__ballot_sync(0xffffffffu, bad)) {
                    err = PARREP_ERANGE;
                    break;
                }
                if (exm) {
                    const unsigned sm = act & ~exm & gm;
                    int src = lane;
                    if (ex) {
                        const int ns = __popc(sm);
                        if (ns > 0) {
                            uint4 w = philox10(make_uint4(r, i, cycle, kTagFV), key);
                            src = kth_set_bit(sm, pick(w.x, (unsigned)ns));
                        } else {
                            src = -1;
                        }
                    }
                    const int s0 = __shfl_sync(0xffffffffu, n0, src < 0 ? lane : src);
                    const int s1 = __shfl_sync(0xffffffffu, n1, src < 0 ? lane : src);
                    if (ex) {
                        n0 = src < 0 ? xt0 : s0;
                        n1 = src < 0 ? xt1 : s1;
                    }
                }
                x0 = n0;
                x1 = n1;
            }
        }
        __syncthreads();
    }
    return err;
}

// Decorrelation of the FP32 form.  Block 0 works in rounds of M = B*RB
// steps: (1) all threads draw the M uniforms; (2) the leader walks the jump
// chain alone -- the states do not depend on the stopping rule, so this
// serial loop carries only the state; (3) all threads turn the states into
// holding times; (4) the leader replays the round in order, applying the
// stopping rule (n_c jumps or t_corr time in W), T_end, T_burn and the
// histogram, and stops where Algorithm 1 stops.  Draws beyond the stop are
// discarded; the next round starts at the step where this one stopped.
template <int KIND>
static __device__ int decorr_chain(const NetDev& N, const FastSmem& F, int x0, int x1, int M, int& last0, int& last1) {
    // (2): states before each of the M jumps; returns the number of jumps
    // made (a jump that leaves [0, hist_max] ends the round, its state is
    // returned in last0/last1)
    const float2* buf = F.buf;
    int* trace = F.trace;
    if (KIND == PARREP_SCHLOGL) {
        // region changes do not stop this chain, only the range does
        const int hm = N.hist_max0;
        int mn = 0, mx = 0;
        int x = x0;
        const int first = spec_pass_schlogl(N, buf, trace, 1, 0, M, 0, hm, x, mn, mx);
        if (first == M) {
            last0 = x;
            last1 = 0;
            return M;
        }
        int y = trace[first];
        for (int k = first; k < M; ++k) {
            trace[k] = y;
            const float4 c = cums_schlogl(N.Af[0], N.Af[1], N.Af[2], N.Af[3], y);
            int J = count_le(c, buf[k].y * c.w);
            if (J == 4) J = last_positive(N, y, 0);
            const int yn = y + ((J & 1) ? -1 : 1);
            if (yn < 0 || yn > hm) {
                last0 = yn;
                last1 = 0;
                return k + 1;
            }
            y = yn;
        }
        last0 = y;
        last1 = 0;
        return M;
    }
    for (int k = 0; k < M; ++k) {
        trace[k] = pack_state(N.nsp, x0, x1);
        const float4 c = cums_f32<KIND>(N, F, x0, x1);
        int J = count_le(c, buf[k].y * c.w);
        if (J == 4) J = last_positive(N, x0, x1);
        int a0 = x0, a1 = x1;
        apply(N, J, a0, a1);
        if (out_of_range(N, a0, a1)) {
            last0 = a0;
            last1 = a1;
            return k + 1;
        }
        x0 = a0;
        x1 = a1;
    }
    last0 = x0;
    last1 = x1;
    return M;
}

// (2) for the Schloegl network with the threshold table, by the whole block,
// in windows of 64 jumps.  From the window's start state x the chain can
// only reach x-64 .. x+64 (129 candidates c, state x + c - 64), and before
// jump s only the candidates with |c - 64| <= s and c - 64 = s (mod 2).
// (a) every reachable (jump, candidate) pair's move is decided from the table
//     in parallel: nx[s][c] = c +- 1;
// (b) each reachable start candidate of each block of 8 jumps is followed
//     through its block: m8[b][c];
// (c) one thread follows the eight block maps from c = 64;
// (d) eight threads walk their block's jumps and write the trace.
// The states are those of the one-thread chain (every choice exact).  A
// window that could reach beyond [0, hist_max] is walked by one thread with
// the range check, and a jump out of the range ends the round (its state in
// last0; returns the number of jumps made).  Called by every thread of the
// block; scratch holds at least 64 * 129 + 8 * 129 bytes.
static __device__ int decorr_chain_block(const NetDev& N, const FastSmem& F, unsigned char* scratch, int x0, int M,
                                         int& last0) {
    __shared__ int s_x, s_n, s_last, s_done;
    __shared__ unsigned char s_bst[8];
    const int tid = threadIdx.x, T = blockDim.x, hm = N.hist_max0;
    unsigned char* nx = scratch;            // [64][129]
    unsigned char* m8 = scratch + 64 * 129;  // [8][129]
    const float2* buf = F.buf;
    int* trace = F.trace;
    if (tid == 0) {
        s_x = x0;
        s_done = 0;
    }
    __syncthreads();
    for (int s0 = 0; s0 < M; s0 += 64) {
        const int x = s_x;
        const int w = min(64, M - s0);
        if (x >= 64 && x + 64 <= hm) {
            // (a) thread -> candidate c and every third reachable jump from its first
            for (int t = tid; t < 3 * 129; t += T) {
                const int c = t % 129, g = t / 129, d = c > 64 ? c - 64 : 64 - c;
                const int4 Tc = F.thr[x + c - 64];
                for (int s = d + 2 * g; s < w; s += 6)
                    nx[s * 129 + c] = (unsigned char)(goes_up_k(Tc, __float_as_int(buf[s0 + s].y)) ? c + 1 : c - 1);
            }
            __syncthreads();
            // (b) items (b, i): block b's reachable start candidates c = 64 - 8b + 2i, i = 0 .. 8b
            for (int t = tid; t < 232; t += T) {
                int b = 0, base = 0;
                while (t >= base + 8 * b + 1) {
                    base += 8 * b + 1;
                    ++b;
                }
                const int c = 64 - 8 * b + 2 * (t - base);
                int y = c;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int s = 8 * b + j;
                    if (s < w) y = nx[s * 129 + y];
                }
                m8[b * 129 + c] = (unsigned char)y;
            }
            __syncthreads();
            // (c) (every thread read s_x before (a)'s barrier); a short last
            // window ends inside block (w - 1) / 8, whose map stops at jump w
            if (tid == 0) {
                int y = 64;
                for (int b = 0; b < 8 && 8 * b < w; ++b) {
                    s_bst[b] = (unsigned char)y;
                    y = m8[b * 129 + y];
                }
                s_x = x + y - 64;
            }
            __syncthreads();
            // (d)
            if (tid < 8) {
                int y = s_bst[tid];
                for (int j = 0; j < 8; ++j) {
                    const int s = 8 * tid + j;
                    if (s < w) {
                        trace[s0 + s] = x + y - 64;
                        y = nx[s * 129 + y];
                    }
                }
            }
            __syncthreads();  // (d) has read nx before the next window writes it
        } else {
            if (tid == 0) {
                int y = x;
                for (int s = 0; s < w; ++s) {
                    trace[s0 + s] = y;
                    const int yn = goes_up_k(F.thr[y], __float_as_int(buf[s0 + s].y)) ? y + 1 : y - 1;
                    if (yn < 0 || yn > hm) {
                        s_n = s0 + s + 1;
                        s_last = yn;
                        s_done = 1;
                        break;
                    }
                    y = yn;
                }
                s_x = y;
            }
            __syncthreads();
            if (s_done) break;
        }
    }
    last0 = s_done ? s_last : s_x;
    const int n = s_done ? s_n : M;
    __syncthreads();  // every thread has read the results before the next round writes them
    return n;
}

// Block-wide exclusive scan of (sum, max) over the threads, in thread order.
__device__ __forceinline__ void block_scan_sum_max(unsigned long long v, int m, unsigned long long* wsum, int* wmax,
                                                   unsigned long long& ex_sum, int& ex_max) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long sv = v;
    int mv = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long su = __shfl_up_sync(0xffffffffu, sv, o);
        const int mu = __shfl_up_sync(0xffffffffu, mv, o);
        if (lane >= o) {
            sv += su;
            mv = max(mv, mu);
        }
    }
    if (lane == 31) {
        wsum[wid] = sv;
        wmax[wid] = mv;
    }
    __syncthreads();
    unsigned long long ws = 0;
    int wm = -1;
    for (int w = 0; w < nw && w < wid; ++w) {
        ws += wsum[w];
        wm = max(wm, wmax[w]);
    }
    const int mprev = __shfl_up_sync(0xffffffffu, mv, 1);
    ex_sum = ws + sv - v;
    ex_max = lane >= 1 ? max(wm, mprev) : wm;
    __syncthreads();
}

// Decorrelation of the FP32 form.  Block 0 works in rounds of M = 4T steps:
// (1) all threads draw the M uniforms; (2) the leader walks the jump chain
// alone -- the only serial part, as the states do not depend on the
// stopping rule; (3) all threads turn the states into holding times; (4) the
// stopping rule (n_c jumps, or t_corr time, of consecutive stay in W), the
// T_end and T_burn crossings are found with block scans -- the in-W counters
// after step k follow from the prefix sums of the holding times and the last
// region change at or before k -- and the committed steps are accumulated in
// parallel.  Draws beyond the stop are discarded; the next round starts at
// the step where this one stopped.
template <int KIND>
static __device__ void decorrelate_f32(const RunParams& P, const FastSmem& F, const HistSink& hs, int sh_post,
                                PhaseClock& pc) {
    __shared__ int s_more, s_n, s_l0, s_l1, s_x0, s_x1, s_W, s_burn, s_status, s_ended;
    __shared__ int s_stop, s_end, s_bcross, s_c, s_M;
    __shared__ long long s_Nc, s_Nc_last;
    __shared__ unsigned long long s_step, s_Ts, s_inW, s_inW_last;
    __shared__ unsigned long long s_wsum[32];
    __shared__ int s_wmax[32];
    __shared__ int s_bmin, s_bmax;
    RunCtl* ctl = P.ctl;
    const NetDev& N = P.net;
    const uint2 key = seed_key(P.seed);
    const unsigned cycle = ldv(&ctl->cycle);
    const bool steps_mode = P.thresh == PARREP_THRESH_STEPS;
    const long long n_c = P.n_c;
    const unsigned long long q_tcorr = P.q_tcorr, q_Tend = P.q_Tend, q_Tburn = P.q_Tburn;
    RegionTest rt0;
    rt0.load(N);
    const int T = blockDim.x, M = min(4 * T, P.B << P.log2RB);  // within buf, trace and decp
    float2* buf = F.buf;
    unsigned long long* qbuf = (unsigned long long*)F.buf;  // (3) overwrites the draws in place
    unsigned long long* Pk = F.decp;                        // inclusive prefix sums of the round
    int* trace = F.trace;
    const bool tabbed = KIND == PARREP_SCHLOGL && F.inv;
    // the block-parallel chain: Schloegl with the threshold table, and the
    // pipelined layout's second and third draw slots as its scratch
    const bool block_chain = KIND == PARREP_SCHLOGL && F.thr != nullptr && P.pipelined;
    unsigned char* chain_scratch = (unsigned char*)(F.buf + (P.B << P.log2RB));
    if (threadIdx.x == 0) {
        s_x0 = ctl->xt0;
        s_x1 = ctl->xt1;
        s_Ts = ctl->Ts;
        s_burn = ctl->burn_done;
        s_W = rt0.region(N.nsp, s_x0, s_x1);
        s_Nc = 0;
        s_inW = 0;
        s_step = 0;
        s_status = 0;
        s_ended = 0;
        s_more = steps_mode ? (0 < n_c) : (0ull < q_tcorr);
    }
    // Round length: M, or -- where the steps the rule still needs can be
    // estimated (STEPS mode; TIME mode with the Schloegl table, as the in-W
    // time still missing times a0 at the current state) -- 1.25 times that
    // plus 64, at least 128, so that the last round draws and walks few steps
    // past the stop.  Rounds never change the results: draws are keyed by
    // the step, and each round starts where the last one stopped.
    auto round_len = [&]() -> int {
        long long est;
        if (steps_mode) est = n_c - s_Nc;
        else if (tabbed && s_inW < q_tcorr) est = (long long)((double)(q_tcorr - s_inW) * 0x1p-40 / (double)F.inv[s_x0]);
        else return M;
        est += est / 4 + 64;
        est = (est + 63) / 64 * 64;  // whole windows of the block chain
        return est < (long long)M ? (int)(est > 128 ? est : 128) : M;
    };
    if (threadIdx.x == 0) s_M = round_len();
    __syncthreads();
    PhaseClock dc{};
    dc.start();
    while (s_more) {
        const unsigned long long step0 = s_step;
        const int Mr = s_M;
        // (1) draws: one Philox call per pair of steps (2p, 2p+1)
        {
            const unsigned long long p0 = step0 >> 1;
            const int npairs = (int)(((step0 + (unsigned long long)Mr - 1) >> 1) - p0) + 1;
            for (int i = threadIdx.x; i < npairs; i += T) {
                const unsigned long long pr = p0 + (unsigned long long)i;
                const uint4 w = philox10(make_uint4((unsigned)(pr >> 32), (unsigned)pr, cycle, kTagDecorr), key);
                const long long ke = (long long)(pr << 1) - (long long)step0;
                // (E, u2), or (E, k2) with k2 the 23-bit index of u2 for the block chain
                const float ya = block_chain ? __int_as_float((int)(w.y >> 9)) : u01f(w.y);
                const float yb = block_chain ? __int_as_float((int)(w.w >> 9)) : u01f(w.w);
                if (ke >= 0 && ke < Mr) buf[ke] = make_float2(-logf(u01f(w.x)), ya);
                if (ke + 1 >= 0 && ke + 1 < Mr) buf[ke + 1] = make_float2(-logf(u01f(w.z)), yb);
            }
        }
        __syncthreads();
        dc.lap(kPhDecDraw);
        // (2) the jump chain
        int bn = 0, bl = 0;
        if (block_chain) bn = decorr_chain_block(N, F, chain_scratch, s_x0, Mr, bl);
        if (threadIdx.x == 0) {
            int l0 = bl, l1 = 0;
            s_n = block_chain ? bn : decorr_chain<KIND>(N, F, s_x0, s_x1, Mr, l0, l1);
            s_l0 = l0;
            s_l1 = l1;
            s_stop = 0x7fffffff;
            s_end = 0x7fffffff;
            s_bcross = 0x7fffffff;
            s_bmin = 0x7fffffff;
            s_bmax = -1;
        }
        __syncthreads();
        dc.lap(kPhDecChain);
        const int n = s_n;
        // (3) holding times
        for (int k = threadIdx.x; k < n; k += T) {
            int a0, a1;
            unpack_state(N.nsp, trace[k], a0, a1);
            const float E = buf[k].x;
            const float ia0 = tabbed ? F.inv[a0] : __frcp_rn(cums_f32<KIND>(N, F, a0, a1).w);
            qbuf[k] = q_of_f32(E * ia0);  // the same thread read buf[k] just before
        }
        __syncthreads();
        dc.lap(kPhDecTimes);
        // (4a) scans: inclusive prefix of q and the last region change
        const int k0 = 4 * threadIdx.x;
        unsigned long long qk[4], lp[4];
        int lc[4], yst[4];
        unsigned long long run = 0;
        int lastc = -1;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + e;
            int a0, a1, y0, y1;
            unpack_state(N.nsp, k < n ? trace[k] : 0, a0, a1);
            if (k + 1 < n) {
                unpack_state(N.nsp, trace[k + 1], y0, y1);
            } else {
                y0 = s_l0;
                y1 = s_l1;
            }
            yst[e] = pack_state(N.nsp, y0, y1);
            qk[e] = k < n ? qbuf[k] : 0ull;
            const bool chg = k < n && !out_of_range(N, y0, y1) &&
                             rt0.region(N.nsp, y0, y1) != rt0.region(N.nsp, a0, a1);
            run += qk[e];
            lp[e] = run;
            if (chg) lastc = k;
            lc[e] = lastc;
        }
        unsigned long long tpre;
        int tmax;
        block_scan_sum_max(run, lastc, s_wsum, s_wmax, tpre, tmax);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (k0 + e < n) Pk[k0 + e] = tpre + lp[e];
        __syncthreads();
        // (4b) the rule before each step, the T_end and T_burn steps
        const unsigned long long Ts0 = s_Ts, inW0 = s_inW;
        const long long Nc0 = s_Nc;
        const int bd0 = s_burn;
        int my_stop = 0x7fffffff, my_end = 0x7fffffff, my_b = 0x7fffffff;
        if (threadIdx.x == 0 && (steps_mode ? (Nc0 >= n_c) : (inW0 >= q_tcorr))) my_stop = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + e;
            if (k >= n) continue;
            const unsigned long long Pe = tpre + lp[e];
            const int L = max(tmax, lc[e]);
            long long Nc;
            unsigned long long inW;
            if (L == k) {
                Nc = 0;
                inW = 0;
            } else if (L < 0) {
                Nc = Nc0 + (long long)(k + 1);
                inW = inW0 + Pe;
            } else {
                Nc = (long long)(k - L);
                inW = Pe - Pk[L];
            }
            if (steps_mode ? (Nc >= n_c) : (inW >= q_tcorr)) my_stop = min(my_stop, k + 1);
            if (Ts0 + Pe >= q_Tend) my_end = min(my_end, k);
            if (!bd0 && Ts0 + Pe >= q_Tburn) my_b = min(my_b, k);
        }
        if (my_stop != 0x7fffffff) atomicMin(&s_stop, my_stop);
        if (my_end != 0x7fffffff) atomicMin(&s_end, my_end);
        if (my_b != 0x7fffffff) atomicMin(&s_bcross, my_b);
        __syncthreads();
        // (4c) commit steps [0, c): c = min(rule stop, T_end step + 1, n)
        const int stop = s_stop, endk = s_end, bk = s_bcross;
        int c = n;
        if (stop < c) c = stop;
        if (endk < c) c = endk + 1;
        const bool ended = endk < n && endk + 1 == c && endk < stop;
        for (int k = threadIdx.x; k < c; k += T) {
            int a0, a1;
            unpack_state(N.nsp, trace[k], a0, a1);
            const unsigned long long Pb = k > 0 ? Pk[k - 1] : 0ull;  // before step k
            const unsigned long long q = Pk[k] - Pb;
            unsigned long long t = q;
            if (ended && k == endk) t = q_Tend - (Ts0 + Pb);
            unsigned long long pre = 0, post = t;
            if (!bd0) {
                if (k < bk) {
                    pre = t;
                    post = 0;
                } else if (k == bk) {
                    const unsigned long long room = q_Tburn - (Ts0 + Pb);
                    pre = t < room ? t : room;
                    post = t - pre;
                }
            }
            if (pre) {
                if (hs.sh && !sh_post) hs.add(a0, a1, pre);
                else atomicAdd(P.hist_pre + a0 * N.ystride + a1, pre);
            }
            if (post) {
                if (hs.sh && sh_post) hs.add(a0, a1, post);
                else atomicAdd(P.hist_post + a0 * N.ystride + a1, post);
            }
            atomicMin(&s_bmin, a0);
            atomicMax(&s_bmax, a0);
        }
        // the carried state after step c-1 (its owner thread writes it)
        if (c > 0 && (c - 1) >= k0 && (c - 1) < k0 + 4) {
            const int e = c - 1 - k0;
            const int k = c - 1;
            const unsigned long long Pe = tpre + lp[e];
            const int L = max(tmax, lc[e]);
            if (L == k) {
                s_Nc_last = 0;
                s_inW_last = 0;
            } else if (L < 0) {
                s_Nc_last = Nc0 + (long long)(k + 1);
                s_inW_last = inW0 + Pe;
            } else {
                s_Nc_last = (long long)(k - L);
                s_inW_last = Pe - Pk[L];
            }
            int y0, y1;
            unpack_state(N.nsp, yst[e], y0, y1);
            s_x0 = y0;
            s_x1 = y1;
            s_c = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int more = 1;
            if (c > 0) {
                s_step = step0 + (unsigned long long)c;
                s_Ts = ended ? q_Tend : Ts0 + Pk[c - 1];
                if (!bd0 && bk < c) s_burn = 1;
                if (ended) {
                    s_ended = 1;
                    more = 0;
                    // the state stays the pre-jump state of the truncated step
                    int a0, a1;
                    unpack_state(N.nsp, trace[endk], a0, a1);
                    s_x0 = a0;
                    s_x1 = a1;
                    s_W = rt0.region(N.nsp, a0, a1);
                } else if (out_of_range(N, s_x0, s_x1)) {
                    // the chain's jump out of range is committed: range error
                    s_status = PARREP_ERANGE;
                    more = 0;
                    int a0, a1;
                    unpack_state(N.nsp, trace[c - 1], a0, a1);
                    s_x0 = a0;
                    s_x1 = a1;
                } else {
                    s_Nc = s_Nc_last;
                    s_inW = s_inW_last;
                    s_W = rt0.region(N.nsp, s_x0, s_x1);
                }
            }
            if (stop <= c) more = 0;  // the rule holds before step c
            if (c < n) more = 0;
            if (n < Mr && c == n && !s_ended && s_status == 0) more = 0;
            atomicAdd(P.progress, 1ull);
            s_more = more;
            if (more) s_M = round_len();
        }
        __syncthreads();
        if (hs.lo && s_bmax >= s_bmin)
            fold_limbs(hs, s_bmin, s_bmax, N.ystride, 0, N.nsp > 1 ? N.hist_max1 : 0);
        __syncthreads();
        dc.lap(kPhDecCommit);
    }
    if (threadIdx.x == 0) {
        for (int i = 8; i < 12; ++i) pc.acc[i] += dc.acc[i];
        leader_finish_decorr(P, s_x0, s_x1, s_W, s_Ts, s_burn, s_step, s_ended != 0, s_status, cycle);
    }
}

// ---------------------------------------------------------------------------
// the persistent ParRep kernel
// ---------------------------------------------------------------------------
// A replay pass (MODE) of the current chunk over this block's virtual
// blocks, each replica from its chunk-start state P.xk.
template <int FORM, int KIND, int MODE>
__device__ __forceinline__ void replay_vblocks(const RunParams& P, const FastSmem& F, const HistSink& hs, int lb,
                                               int nblk, int nvb, const RegionTest& rt, unsigned cycle, unsigned n0, int S,
                                               uint2 key,
                                               const Cuts& cut, bool to_post, unsigned long long& ev_replay,
                                               PhaseClock& pc, unsigned long long* inc_q = nullptr,
                                               unsigned long long* inc_ev = nullptr) {
    const bool owner = (int)threadIdx.x < P.RB;
    for (int vb = lb; vb < nvb; vb += nblk) {
        const unsigned rbase = (unsigned)vb * (unsigned)P.RB, r = rbase + threadIdx.x;
        const bool active = owner && (long long)r < (long long)P.R;
        int y0 = 0, y1 = 0;
        if (active) {
            const int2 xv = P.xk[r];
            y0 = xv.x;
            y1 = xv.y;
        }
        unsigned long long d0 = 0, d1 = 0;
        unsigned long long& q = MODE == kPrecise ? *inc_q : d0;
        unsigned long long& e = MODE == kPrecise ? *inc_ev : d1;
        if (FORM == kFormF32Staged) {
            unsigned long long k0 = kNone, k1 = kNone;
            int e0 = 0, e1 = 0;
            chunk_f32<KIND, MODE>(P, F, hs, active, rbase, r, rt, cycle, n0, S, key, y0, y1, cut, to_post, k0, k1, e0,
                                  e1, q, ev_replay, e, pc);
        } else if (MODE == kStepSum) {
            // whole warps of owner threads (RB is a multiple of 32)
            if (owner) replay_stepsum_warp<FORM != kFormF64>(P, active, y0, y1, r, rt.W, cycle, n0, S, cut, ev_replay);
        } else if (active) {
            replay_chunk<FORM != kFormF64, MODE>(P, hs, y0, y1, r, rt.W, cycle, n0, S, cut, to_post, q, e, ev_replay);
        }
    }
}

// The whole block: the first index k of v[0..n) with base + v[0] + ... + v[k]
// >= target (fixed-point holding times), and part = target - (base + v[0] +
// ... + v[k-1]), the share of v[k] before the threshold; -1 if the sums stay
// below it.  Chunks of blockDim.x values: a warp scan by shuffles, a scan of
// the warp totals, and the smallest crossing index by a shared atomic min --
// the same k and part as a serial scan, in about n / blockDim.x rounds.
static __device__ int block_find_crossing(const unsigned long long* __restrict__ v, int n, unsigned long long base,
                                          unsigned long long target, unsigned long long& part) {
    __shared__ unsigned long long s_w[33];
    __shared__ int s_k;
    __shared__ unsigned long long s_part;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    unsigned long long acc = base;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const unsigned long long x = i < n ? __ldcg(v + i) : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        if (threadIdx.x == 0) s_k = 0x7fffffff;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < nw; ++w) {
                const unsigned long long a = s_w[w];
                s_w[w] = t;  // exclusive prefix of the warp totals
                t += a;
            }
            s_w[32] = t;     // the chunk's total
        }
        __syncthreads();
        const unsigned long long incl = acc + s_w[warp] + inc;
        if (i < n && incl >= target) atomicMin(&s_k, i);
        __syncthreads();
        const int k = s_k;
        if (k != 0x7fffffff) {
            if (i == k) s_part = target - (incl - x);
            __syncthreads();
            part = s_part;
            __syncthreads();
            return k;
        }
        acc += s_w[32];
        __syncthreads();
    }
    part = 0;
    return -1;
}

// Batches: at the start of a cycle the instance's leader thread claims idle
// blocks (up to one block per group of replicas) and posts each its place in
// the gang; the joiners start with the dephasing, after the barrier that
// ends this cycle's decorrelation.  Also publishes what a joiner needs to
// stay in step (chunk count, last chunk's sums).
static __device__ void recruit(const RunParams& P, RunCtl* ctl, int nblk, int nvb, unsigned long long chunk_c,
                        unsigned long long est_q, unsigned long long est_ev) {
    ctl->chunk_c = chunk_c;
    ctl->est_q = est_q;
    ctl->est_ev = est_ev;
    const unsigned gen = ldv(&ctl->bar_gen);
    constexpr int kMaxRecruit = 128;
    int want = min(nvb - nblk, kMaxRecruit);
    int got = 0;
    const int nw = ((int)gridDim.x + 31) / 32;
    if (want > 0 && (P.batch.reserve > 0 || P.batch.tail)) {
        // serving: leave the reserve and one idle block for every request
        // that is published and not yet claimed
        int idle = 0;
        for (int w = 0; w < nw; ++w) idle += __popc(ldv(&P.batch.idle[w]));
        long long pending = 0;
        if (P.batch.tail) pending = (long long)(ld_acquire_sys(P.batch.tail) - ldv(P.batch.head));
        want = (int)min((long long)want, (long long)idle - P.batch.reserve - pending);
    }
    short ids[kMaxRecruit];
    for (int w = 0; w < nw && got < want; ++w) {
        unsigned m = ldv(&P.batch.idle[w]);
        while (m && got < want) {
            const unsigned bit = m & (0u - m);
            m &= ~bit;
            const unsigned old = atomicAnd(&P.batch.idle[w], ~bit);
            if (old & bit) ids[got++] = (short)(w * 32 + (__ffs(bit) - 1));
        }
    }
    // the gang size first, so that no member can ever see a smaller one
    ctl->nblk = nblk + got;
    __threadfence();
    for (int j = 0; j < got; ++j) {
        int4* mb = &P.batch.mail[ids[j]];
        ((volatile int*)mb)[0] = P.inst;
        ((volatile int*)mb)[1] = nblk + j;
        ((volatile int*)mb)[2] = (int)gen;
        __threadfence();
        atomicExch(&mb->w, 1);
    }
}

// A joiner waits (bounded) until the barrier of generation gen has passed.
static __device__ bool wait_generation(const RunParams& P, RunCtl* ctl, unsigned gen) {
    unsigned long long t0 = globaltimer(), p0 = ldv(P.progress);
    unsigned ns = 32;
    while (ldv(&ctl->bar_gen) == gen) {
        if (ldv(&ctl->status) != 0) return false;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        const unsigned long long p = ldv(P.progress), t = globaltimer();
        if (p != p0) {
            p0 = p;
            t0 = t;
        } else if ((long long)(t - t0) > P.timeout_ns) {
            atomicCAS(&ctl->status, 0, PARREP_ETIMEOUT);
            return false;
        }
    }
    __threadfence();
    return true;
}

// One ParRep run (Algorithm 1) of the instance P by the P.nblk blocks that
// serve it; lb is this block's index among them.  Replicas come in virtual
// blocks of RB (vb = 0 .. ceil(R / RB) - 1); block lb takes vb = lb,
// lb + nblk, ...  A replica's state lives in P.xs between the phases (and
// its chunk-start state in P.xk, its exit state in P.xe), so an instance can
// have more replicas than its blocks have owner threads.  Lockstep is logical:
// each replica takes the same steps whatever block takes it and in whatever
// order, so every result is independent of nblk.
template <int FORM, int KIND>
__device__ __forceinline__ bool run_instance(const RunParams& P, int lb, unsigned char* smem, BlockScratch& red,
                                             int join_gen = -1) {
    constexpr bool F32 = FORM != kFormF64;           // binary32 propensities and selection
    constexpr bool STAGED = FORM == kFormF32Staged;  // owner threads + helper warps
    RunCtl* ctl = P.ctl;
    const NetDev& N = P.net;
    const bool batch = P.batch.remaining != nullptr;
    const bool join = join_gen >= 0;  // a block recruited at a cycle start
    int nblk = P.nblk;
    const int nvb = (P.R + P.RB - 1) / P.RB;
    const bool owner = (int)threadIdx.x < P.RB;
    const bool leader = lb == 0 && threadIdx.x == 0;
    const uint2 key = seed_key(P.seed);
    unsigned long long* sh_hist = (unsigned long long*)smem;
    BarState bs{0, lb, nblk};
    PhaseClock pc{};
    FastSmem F{};
    unsigned* limb_lo = nullptr;
    unsigned* limb_hi = nullptr;
    if (STAGED) {
        if (P.use_smem_hist) {
            limb_lo = (unsigned*)(smem + P.off_limbs);
            limb_hi = limb_lo + N.nbins;
            for (int b = threadIdx.x; b < 2 * N.nbins; b += blockDim.x) limb_lo[b] = 0;
        }
        F.inv = P.off_inv >= 0 && KIND == PARREP_SCHLOGL ? (const float*)(smem + P.off_inv) : nullptr;
        F.thr = P.off_thr >= 0 && KIND == PARREP_SCHLOGL ? (const int4*)(smem + P.off_thr) + kThrPad : nullptr;
        F.rng = (int*)(smem + P.off_rng);
        F.decp = (unsigned long long*)(smem + P.off_decp);
        F.prodU = KIND == PARREP_TOGGLE ? (const float*)(smem + P.off_tab) : nullptr;
        F.prodV = KIND == PARREP_TOGGLE ? (const float*)(smem + P.off_tab) + (N.hist_max1 + 1) : nullptr;
        F.buf = (float2*)(smem + P.off_buf);
        F.trace = (int*)(smem + P.off_trace);
        F.live = (int*)(smem + P.off_live);
        F.nvalid = (int*)(smem + P.off_nvalid);
        build_fast_tables(N, (float*)F.inv, (float*)F.prodU, (float*)F.prodV);
        if (KIND == PARREP_SCHLOGL && F.thr) build_thr_table(N, (int4*)F.thr);
    }

    if (P.use_smem_hist) {
        for (int b = threadIdx.x; b < N.nbins; b += blockDim.x) sh_hist[b] = 0;
    }
    unsigned long long ev_replay = 0;

    if (leader && !join) {
        int x0 = P.x00, x1 = P.x01;
        if (P.x0_hi > 0) {
            uint4 w = philox10(make_uint4(0u, 0u, 0u, kTagInit), key);
            x0 = (int)pick(w.x, (unsigned)P.x0_hi + 1u);
            x1 = N.nsp > 1 ? (int)pick(w.y, (unsigned)P.x0_hi + 1u) : 0;
        }
        ctl->x00 = x0;
        ctl->x01 = x1;
        ctl->xt0 = x0;
        ctl->xt1 = x1;
        ctl->Ts = 0;
        ctl->cycle = 0;
        ctl->burn_done = P.q_Tburn == 0 ? 1 : 0;
        ctl->W = region_of(N, x0, x1);
        if (out_of_range(N, x0, x1)) atomicCAS(&ctl->status, 0, PARREP_EINVAL);
        ctl->done = P.q_Tend == 0 ? 1 : 0;
        ctl->nblk = nblk;
        for (int s = 0; s < 3; ++s) {
            ctl->minkey[s] = kNone;
            ctl->oobkey[s] = kNone;
            ctl->chunksum[s] = 0;
            ctl->chunkev[s] = 0;
            ctl->inc_sum[s] = 0;
            ctl->inc_ev[s] = 0;
        }
        __threadfence();
    }
    int period_post = P.q_Tburn == 0 ? 1 : 0;  // which global sums this block's histogram feeds
    HistSink hs{P.use_smem_hist ? sh_hist : nullptr, period_post ? P.hist_post : P.hist_pre, limb_lo, limb_hi,
                N.ystride,
                STAGED ? (1ull << 47) / ((unsigned long long)P.B * (unsigned long long)P.RB *
                                         (unsigned long long)fold_period(P.B, P.log2RB))
                       : 0ull};
    unsigned long long chunk_c = 0;
    unsigned long long est_q = 0, est_ev = 0;  // time and jumps of the last chunk
    if (join) {
        __shared__ int s_ok;
        if (threadIdx.x == 0) s_ok = wait_generation(P, ctl, (unsigned)join_gen) ? 1 : 0;
        __syncwarp();
        __syncthreads();
        if (!s_ok) goto out;
        nblk = ldv(&ctl->nblk);
        bs.nblk = nblk;
        chunk_c = ldv(&ctl->chunk_c);
        est_q = ldv(&ctl->est_q);
        est_ev = ldv(&ctl->est_ev);
        if (ldv(&ctl->burn_done) && !period_post) {
            period_post = 1;
            hs.g = P.hist_post;
        }
    } else if (!grid_sync(P, bs)) {
        goto out;
    }

    for (bool first = true;; first = false) {
        // ---------------- decorrelation (serial) ----------------
        // (a block that joined at this cycle's start begins after it)
        if (!(join && first)) {
            pc.start();
            if (STAGED) {
                if (lb == 0 && !ldv(&ctl->done))
                    decorrelate_f32<KIND>(P, F, hs, period_post, pc);
            } else {
                if (leader && !ctl->done) leader_decorrelate<F32>(P);
            }
            if (batch && leader && !ldv(&ctl->done)) recruit(P, ctl, nblk, nvb, chunk_c, est_q, est_ev);
            pc.lap(kPhDecorr);
            if (!grid_sync(P, bs)) goto out;
            pc.lap(kPhBarrier);
            if (batch) {
                nblk = ldv(&ctl->nblk);
                bs.nblk = nblk;
            }
            if (ldv(&ctl->done)) break;
        }
        {
            const int W = ldv(&ctl->W);
            RegionTest rt;
            rt.init(N, W);
            const int xt0 = ldv(&ctl->xt0), xt1 = ldv(&ctl->xt1);
            const long long np = ldv(&ctl->np);
            const unsigned cycle = ldv(&ctl->cycle);
            unsigned long long Ts = ldv(&ctl->Ts);
            int burn_done = ldv(&ctl->burn_done);
            if (burn_done && !period_post) {
                if (hs.sh) flush_shared(sh_hist, P.hist_pre, N.nbins);
                period_post = 1;
                hs.g = P.hist_post;
            }
            // ---------------- dephasing ----------------
            pc.start();
            {
                int derr = 0;
                for (int vb = lb; vb < nvb; vb += nblk) {
                    const unsigned rbase = (unsigned)vb * (unsigned)P.RB, r = rbase + threadIdx.x;
                    const bool active = owner && (long long)r < (long long)P.R;
                    int x0, x1;
                    if (STAGED) derr |= dephase_f32<KIND>(P, F, rt, active, rbase, r, xt0, xt1, np, cycle, key, x0, x1);
                    else derr |= dephase_warp<F32>(N, active, r, P.G, W, xt0, xt1, np, cycle, key, x0, x1);
                    if (active) P.xs[r] = make_int2(x0, x1);
                    __syncwarp();
                    __syncthreads();
                }
                if (derr && (threadIdx.x & 31) == 0) atomicCAS(&ctl->status, 0, PARREP_ERANGE);
            }
            pc.lap(kPhDephase);
            if (leader) ctl->ev_dephase += (unsigned long long)np * (unsigned long long)P.R;
            // ---------------- parallel step ----------------
            unsigned n0 = 0;
            int grow = 0;
            for (;;) {
                // chunk length: doubling from one sub-chunk at the start of a
                // cycle up to P.S.  When the next threshold (T_burn, T_end) is
                // within reach, by the last chunk's time per lockstep step, the
                // chunk stops short of it (L - 0.1 L - unit/2 steps of the L
                // estimated to be left, rounded down to whole sub-chunks): it is
                // committed without a replay, and only the short chunk that
                // crosses the threshold (at most 1.25 L + 1 steps) is replayed.
                // Every block computes it from the same values; results do not
                // depend on where chunks end.
                int Sc = P.S;
                {
                    const int unit = STAGED ? P.B : 32;
                    if (grow < 30 && ((long long)unit << grow) < (long long)Sc) Sc = unit << grow;
                    const unsigned long long q_lim = burn_done ? P.q_Tend : P.q_Tburn;
                    if (est_ev > 0 && est_q > 0 && q_lim > Ts) {
                        const double step_q = (double)est_q * (double)P.R / (double)est_ev;
                        const double left = (double)(q_lim - Ts) / step_q;
                        const double need = ceil(left * 1.25) + 1.0;
                        if (need < (double)Sc) {
                            const double lead = left - (0.1 * left + 0.5 * unit);
                            int nd = lead >= (double)unit ? (int)lead / unit * unit
                                                          : ((int)need + unit - 1) / unit * unit;
                            Sc = nd < unit ? unit : nd;
                        }
                    }
                    ++grow;
                }
                if ((unsigned long long)n0 + (unsigned long long)Sc > 0xFFFFFFFFull) {
                    if (leader) atomicCAS(&ctl->status, 0, PARREP_ERANGE);
                }
                if (leader) {
                    const int s1 = (int)((chunk_c + 1) % 3);
                    ctl->minkey[s1] = kNone;
                    ctl->oobkey[s1] = kNone;
                    ctl->chunksum[s1] = 0;
                    ctl->chunkev[s1] = 0;
                    ctl->inc_sum[s1] = 0;
                    ctl->inc_ev[s1] = 0;
                }
                __syncwarp();  // the leader's lanes meet again before the block-wide chunk
                unsigned long long mykey = kNone, myoob = kNone, qsum = 0, ev = 0;
                Cuts none{kNone, kNone, kNone, 0, kNone, 0, -1, -1};
                if (!STAGED) pc.start();  // the staged chunks time their own stages
                for (int vb = lb; vb < nvb; vb += nblk) {
                    const unsigned rbase = (unsigned)vb * (unsigned)P.RB, r = rbase + threadIdx.x;
                    const bool active = owner && (long long)r < (long long)P.R;
                    int x0 = 0, x1 = 0, xe0 = 0, xe1 = 0;
                    if (active) {
                        const int2 xv = P.xs[r];
                        x0 = xv.x;
                        x1 = xv.y;
                        P.xk[r] = xv;
                    }
                    unsigned long long k0 = kNone, k1 = kNone;
                    if (STAGED) {
                        unsigned long long dummy = 0;
                        chunk_f32<KIND, kFirst>(P, F, hs, active, rbase, r, rt, cycle, n0, Sc, key, x0, x1, none,
                                                period_post, k0, k1, xe0, xe1, qsum, ev, dummy, pc);
                    } else if (active) {
                        uint4 wp = make_uint4(0u, 0u, 0u, 0u);
                        for (int s = 0; s < Sc; ++s) {
                            // binary32: one Philox call per step pair (n0 is even)
                            const unsigned n = n0 + (unsigned)s;
                            uint4 w;
                            if (F32) {
                                if ((n & 1u) == 0u) wp = philox10(make_uint4(r, n >> 1, cycle, kTagParallel), key);
                                w = (n & 1u) ? make_uint4(wp.z, wp.w, 0u, 0u) : wp;
                            } else {
                                w = par_words<F32>(r, n, cycle, key);
                            }
                            unsigned long long q = 0;
                            const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
                            qsum += q;
                            ++ev;
                            hs.add(x0, x1, q);
                            int a0 = x0, a1 = x1;
                            apply(N, J, a0, a1);
                            if (out_of_range(N, a0, a1)) {
                                k1 = pos_of(s, r);
                                break;
                            }
                            if (region_of(N, a0, a1) != W) {
                                k0 = pos_of(s, r);
                                xe0 = a0;
                                xe1 = a1;
                                break;
                            }
                            x0 = a0;
                            x1 = a1;
                        }
                    }
                    if (active) {
                        P.xs[r] = make_int2(x0, x1);
                        if (k0 != kNone) P.xe[r] = make_int2(xe0, xe1);
                    }
                    mykey = k0 < mykey ? k0 : mykey;
                    myoob = k1 < myoob ? k1 : myoob;
                }
                const int slot = (int)(chunk_c % 3);
                if (!STAGED) pc.lap(kPhChain);
                pc.start();
                {
                    unsigned long long a = mykey, b = myoob, c = qsum, d = ev;
                    block_reduce4(red, a, b, c, d);
                    if (threadIdx.x == 0) {
                        if (a != kNone) atomicMin(&ctl->minkey[slot], a);
                        if (b != kNone) atomicMin(&ctl->oobkey[slot], b);
                        if (c) atomicAdd(&ctl->chunksum[slot], c);
                        if (d) atomicAdd(&ctl->chunkev[slot], d);
                    }
                }
                pc.lap(kPhVote);
                if (!grid_sync(P, bs)) goto out;
                pc.lap(kPhBarrier);
                ++chunk_c;
                const unsigned long long ekey = ldv(&ctl->minkey[slot]);
                const unsigned long long okey = ldv(&ctl->oobkey[slot]);
                const unsigned long long csum = ldv(&ctl->chunksum[slot]);
                const unsigned long long cev = ldv(&ctl->chunkev[slot]);
                const unsigned long long q_next = burn_done ? P.q_Tend : P.q_Tburn;
                if (cev > 0 && csum > 0) {
                    est_q = csum;
                    est_ev = cev;
                }
                if (leader) {
                    ctl->chunks += 1;
                    ctl->ev_par_exec += cev;
                }
                if (ekey == kNone && okey == kNone && Ts + csum < q_next) {
                    Ts += csum;
                    if (leader) {
                        ctl->ev_useful += cev;
                        ctl->Ts = Ts;
                    }
                    n0 += (unsigned)Sc;
                    continue;
                }
                // ------------- special chunk: escape, range error or time cut -------------
                if (leader) ctl->special += 1;
                __syncwarp();
                pc.start();
                replay_vblocks<FORM, KIND, kRollback>(P, F, hs, lb, nblk, nvb, rt, cycle, n0, Sc, key, none, period_post,
                                                     ev_replay, pc);
                Cuts cut{kNone, kNone, kNone, 0, kNone, 0, -1, -1};
                cut.posE = ekey;
                cut.posC = ekey < okey ? ekey : okey;
                if (Ts + csum >= q_next) {
                    // a threshold may be crossed: find the step, then the replica
                    if (lb == 0) {
                        for (int j = threadIdx.x; j < Sc; j += blockDim.x) P.step_sum[j] = 0;
                    }
                    if (!grid_sync(P, bs)) goto out;
                    replay_vblocks<FORM, KIND, kStepSum>(P, F, hs, lb, nblk, nvb, rt, cycle, n0, Sc, key, cut, period_post,
                                                        ev_replay, pc);
                    if (!grid_sync(P, bs)) goto out;
                    unsigned long long baseB = 0, baseT = 0;
                    {
                        unsigned long long acc = Ts;
                        for (int j = 0; j < Sc; ++j) {
                            const unsigned long long v = __ldcg(P.step_sum + j);
                            if (!burn_done && cut.nB < 0 && acc + v >= P.q_Tburn) {
                                cut.nB = j;
                                baseB = acc;
                            }
                            if (cut.nT < 0 && acc + v >= P.q_Tend) {
                                cut.nT = j;
                                baseT = acc;
                            }
                            acc += v;
                        }
                    }
                    if (cut.nB >= 0 || cut.nT >= 0) {
                        for (int vb = lb; vb < nvb; vb += nblk) {
                            const unsigned r = (unsigned)vb * (unsigned)P.RB + threadIdx.x;
                            if (owner && (long long)r < (long long)P.R) {
                                P.tau_at[r] = 0;
                                P.tau_at[P.R + r] = 0;
                            }
                        }
                        replay_vblocks<FORM, KIND, kTauAt>(P, F, hs, lb, nblk, nvb, rt, cycle, n0, Sc, key, cut, period_post,
                                                          ev_replay, pc);
                        if (!grid_sync(P, bs)) goto out;
                        if (lb == 0) {
                            // block 0 finds the replicas whose holding time at the
                            // crossing step crosses T_burn / T_end: the first rr with
                            // base + sum_{i <= rr} tau_i >= the threshold, by a
                            // block-parallel prefix scan over the replicas
                            __syncwarp();
                            int kB = -1, kT = -1;
                            unsigned long long partB = 0, partT = 0;
                            if (cut.nB >= 0) kB = block_find_crossing(P.tau_at, P.R, baseB, P.q_Tburn, partB);
                            if (cut.nT >= 0) kT = block_find_crossing(P.tau_at + P.R, P.R, baseT, P.q_Tend, partT);
                            if (threadIdx.x == 0) {
                                ctl->posB = kB >= 0 ? pos_of(cut.nB, (unsigned)kB) : kNone;
                                ctl->partB = partB;
                                ctl->posT = kT >= 0 ? pos_of(cut.nT, (unsigned)kT) : kNone;
                                ctl->partT = partT;
                                __threadfence();
                            }
                        }
                        if (!grid_sync(P, bs)) goto out;
                        cut.posB = ldv(&ctl->posB);
                        cut.partB = ldv(&ctl->partB);
                        cut.posT = ldv(&ctl->posT);
                        cut.partT = ldv(&ctl->partT);
                    }
                }
                // a range error stands if the replica's jump really happened
                if (okey != kNone && okey <= cut.posE && okey < cut.posT) {
                    if (leader) atomicCAS(&ctl->status, 0, PARREP_ERANGE);
                    grid_sync(P, bs);
                    goto out;
                }
                if (cut.posB != kNone) {
                    // this block's shared sums are all before T_burn now; what
                    // the precise pass adds to the sink is after it
                    if (hs.sh) flush_shared(sh_hist, P.hist_pre, N.nbins);
                    hs.g = P.hist_post;
                }
                {
                    unsigned long long inc_q = 0, inc_ev = 0;
                    const bool tp = period_post || cut.posB != kNone;
                    replay_vblocks<FORM, KIND, kPrecise>(P, F, hs, lb, nblk, nvb, rt, cycle, n0, Sc, key, cut, tp, ev_replay,
                                                        pc, &inc_q, &inc_ev);
                    unsigned long long a = kNone, b = kNone;
                    block_reduce4(red, a, b, inc_q, inc_ev);
                    if (threadIdx.x == 0) {
                        if (inc_q) atomicAdd(&ctl->inc_sum[slot], inc_q);
                        if (inc_ev) atomicAdd(&ctl->inc_ev[slot], inc_ev);
                    }
                }
                if (cut.posB != kNone) {
                    burn_done = 1;
                    period_post = 1;
                    hs.g = P.hist_post;
                }
                pc.lap(kPhSpecial);
                if (!grid_sync(P, bs)) goto out;
                pc.lap(kPhBarrier);
                Ts += ldv(&ctl->inc_sum[slot]);
                const bool t_end = cut.posT != kNone && cut.posT <= cut.posE;
                if (leader) {
                    ctl->ev_useful += ldv(&ctl->inc_ev[slot]);
                    ctl->Ts = Ts;
                    ctl->burn_done = burn_done;
                    CycleRecDev rec{};
                    const long long i = ctl->log_n;
                    if (i < P.log_cap) rec = P.log[i];
                    if (t_end || ekey != kNone) {
                        rec.ended = t_end ? 1 : 0;
                        rec.n_star = (long long)n0 + (long long)((t_end ? cut.posT : ekey) >> 32) + 1;
                        rec.k = t_end ? -1 : (long long)(ekey & 0xffffffffu);
                        if (!t_end) {
                            // the escaping replica's X^K_{N*}, written in the first pass
                            const int2 xe = __ldcg(P.xe + (ekey & 0xffffffffu));
                            ctl->xt0 = xe.x;
                            ctl->xt1 = xe.y;
                            ctl->escapes += 1;
                        }
                        rec.xt0 = ctl->xt0;
                        rec.xt1 = ctl->xt1;
                        rec.Ts = t_end ? P.q_Tend : Ts;
                        if (t_end) ctl->Ts = P.q_Tend;
                        leader_log(P, ctl, rec);
                        ctl->cycles += 1;
                        ctl->cycle = cycle + 1;
                        if (t_end) ctl->done = 1;
                    }
                    __threadfence();
                }
                if (t_end) goto finished;
                if (ekey != kNone) break;  // next cycle
                n0 += (unsigned)Sc;        // only the T_burn split was in this chunk
            }
        }
        if (!grid_sync(P, bs)) goto out;
    }
finished:
out:
    if (P.use_smem_hist) flush_shared(sh_hist, period_post ? P.hist_post : P.hist_pre, N.nbins);
    {
        unsigned long long a = kNone, b = kNone, c = ev_replay, d = 0;
        block_reduce4(red, a, b, c, d);
        if (threadIdx.x == 0 && c) atomicAdd(&ctl->ev_replay, c);
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 12; ++i)
            if (pc.acc[i]) atomicAdd(&ctl->phase_cycles[i], pc.acc[i]);
    if (batch && leader) {
        __threadfence();
        atomicSub(P.batch.remaining, 1);
    }
    // the last block of the gang to leave (for an epilogue after all flushes)
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&ctl->exited, 1u);
        __threadfence();
        const bool over = ldv(&ctl->done) != 0 || ldv(&ctl->status) != 0;
        s_last = over && old + 1 == (unsigned)ldv(&ctl->nblk) ? 1 : 0;
    }
    __syncwarp();
    __syncthreads();
    return s_last != 0;
}

// One instance on the whole grid.
// Launch bounds per form: the binary32 direct form runs kDirectThreads
// threads per block with kDirectMinBlocks blocks per SM (one thread per
// replica at high occupancy); the others up to kMaxThreads with one block.
#define PARREP_BOUNDS(FORM) \
    __launch_bounds__((FORM) == kFormF32Direct ? kDirectThreads : kMaxThreads, \
                      (FORM) == kFormF32Direct ? kDirectMinBlocks : 1)

template <int FORM, int KIND>
__global__ void PARREP_BOUNDS(FORM) parrep_run_kernel(RunParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockScratch red;
    run_instance<FORM, KIND>(P, (int)blockIdx.x, smem, red);
}

// Many instances in one persistent launch.  Block b works through its list
// items[off[b] .. off[b+1]) of (instance, local block index); the blocks that
// serve an instance (its gang, P.nblk of them at the start) meet at its
// barriers.  The host orders every list by the instances' start times in one
// schedule, so any two blocks meet their shared instances in the same order
// and no wait is circular.  A block whose list is done goes idle: it sets its
// bit in bd.idle and waits (bounded, on the batch's progress) for a mailbox
// entry from an instance that recruits it at a cycle start, until no
// instance is left.  Both network kinds run in the same launch.
// One instance in a batch or serve kernel of the given form; the mixed form
// runs each instance in the binary32 layout its parameters name (P.form).
// The genetic switch runs in the two-species instantiation.
template <int FORM>
__device__ __forceinline__ bool run_any(const RunParams& P, int lb, unsigned char* smem, BlockScratch& red,
                                        int join_gen) {
    if constexpr (FORM == kFormF32Mixed) {
        if (P.form == kFormF32Direct)
            return P.net.kind == PARREP_SCHLOGL ? run_instance<kFormF32Direct, PARREP_SCHLOGL>(P, lb, smem, red, join_gen)
                                                : run_instance<kFormF32Direct, PARREP_TOGGLE>(P, lb, smem, red, join_gen);
        return P.net.kind == PARREP_SCHLOGL ? run_instance<kFormF32Staged, PARREP_SCHLOGL>(P, lb, smem, red, join_gen)
                                            : run_instance<kFormF32Staged, PARREP_TOGGLE>(P, lb, smem, red, join_gen);
    } else {
        return P.net.kind == PARREP_SCHLOGL ? run_instance<FORM, PARREP_SCHLOGL>(P, lb, smem, red, join_gen)
                                            : run_instance<FORM, PARREP_TOGGLE>(P, lb, smem, red, join_gen);
    }
}

template <int FORM>
__device__ __forceinline__ void batch_item(const RunParams* Ps, RunParams& sP, int inst, int lb, int join_gen,
                                           unsigned char* smem, BlockScratch& red) {
    const int* src = (const int*)(Ps + inst);
    int* dst = (int*)&sP;
    for (int w = threadIdx.x; w < (int)(sizeof(RunParams) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    run_any<FORM>(sP, lb, smem, red, join_gen);
    __syncthreads();
}

template <int FORM>
__global__ void PARREP_BOUNDS(FORM)
    parrep_batch_kernel(const RunParams* __restrict__ Ps, const int* __restrict__ off,
                        const int2* __restrict__ items, BatchDev bd) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockScratch red;
    __shared__ RunParams sP;
    __shared__ int4 s_mail;
    const int k1 = off[blockIdx.x + 1];
    for (int k = off[blockIdx.x]; k < k1; ++k) {
        const int2 it = items[k];
        batch_item<FORM>(Ps, sP, it.x, it.y, -1, smem, red);
    }
    // idle: offer this block to instances that start a cycle
    const unsigned long long* progress = Ps[0].progress;
    const long long timeout_ns = Ps[0].timeout_ns;
    int4* mb = bd.mail + blockIdx.x;
    unsigned* word = bd.idle + blockIdx.x / 32;
    const unsigned bit = 1u << (blockIdx.x % 32);
    for (;;) {
        if (threadIdx.x == 0) {
            int4 m = make_int4(-1, 0, 0, 0);
            ((volatile int*)mb)[3] = 0;
            __threadfence();
            atomicOr(word, bit);
            unsigned long long t0 = globaltimer(), p0 = ldv(progress);
            unsigned ns = 64;
            bool got = false;
            for (;;) {
                if (ldv(&mb->w)) {
                    got = true;
                    break;
                }
                if (ldv(bd.remaining) <= 0) break;
                __nanosleep(ns);
                if (ns < 2048) ns <<= 1;
                const unsigned long long p = ldv(progress), t = globaltimer();
                if (p != p0) {
                    p0 = p;
                    t0 = t;
                } else if ((long long)(t - t0) > timeout_ns) {
                    break;
                }
            }
            if (!got) {
                // withdraw; if an instance claimed the block meanwhile, its
                // mail follows the claim at once
                const unsigned old = atomicAnd(word, ~bit);
                if (!(old & bit)) {
                    const unsigned long long t1 = globaltimer();
                    while (!ldv(&mb->w) && (long long)(globaltimer() - t1) < timeout_ns) __nanosleep(64);
                    got = ldv(&mb->w) != 0;
                }
            }
            if (got) {
                __threadfence();
                m = make_int4(ldv(&mb->x), ldv(&mb->y), ldv(&mb->z), 1);
            }
            s_mail = m;
        }
        __syncwarp();
        __syncthreads();
        const int4 m = s_mail;
        __syncthreads();
        if (m.x < 0) break;
        batch_item<FORM>(Ps, sP, m.x, m.y, m.z, smem, red);
    }
}

// ---------------------------------------------------------------------------
// serving: requests from a host-mapped ring, continuous batching
// ---------------------------------------------------------------------------

// What a serving block does next (thread 0): join a gang that recruited it
// (w = 2: slot, block index, barrier generation), lead a newly published
// request (w = 1: slot), or leave (w = 0) on the stop flag, or once the
// whole server has had nothing published and nothing in flight for
// idle_exit_ns (a block never leaves while others still serve requests, so
// the launch keeps all its blocks until it ends).  While it waits it is in
// the idle set.
static __device__ int4 serve_next(const ServeDev& sd) {
    int4* mb = sd.bd.mail + blockIdx.x;
    unsigned* word = sd.bd.idle + blockIdx.x / 32;
    const unsigned bit = 1u << (blockIdx.x % 32);
    ((volatile int*)mb)[3] = 0;
    __threadfence();
    atomicOr(word, bit);
    unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        if (ldv(&mb->w)) {
            __threadfence();
            return make_int4(ldv(&mb->x), ldv(&mb->y), ldv(&mb->z), 2);
        }
        const unsigned long long tail = ld_acquire_sys(sd.tail);
        const unsigned long long head = ldv(sd.head);
        const bool stop = ld_acquire_sys(sd.stop) != 0;
        const bool busy = head < tail || ldv(sd.finished) < head;
        if (busy) t0 = globaltimer();
        const bool idle_out = (long long)(globaltimer() - t0) > sd.idle_exit_ns;
        if (head < tail || stop || idle_out) {
            const unsigned old = atomicAnd(word, ~bit);
            if (!(old & bit)) {
                // a gang claimed this block meanwhile: its mail follows at once
                const unsigned long long t1 = globaltimer();
                while (!ldv(&mb->w) && (long long)(globaltimer() - t1) < 1000000000ll) __nanosleep(64);
                if (!ldv(&mb->w)) return make_int4(0, 0, 0, 0);
                __threadfence();
                return make_int4(ldv(&mb->x), ldv(&mb->y), ldv(&mb->z), 2);
            }
            if (stop || (head >= tail && idle_out)) return make_int4(0, 0, 0, 0);
            if (head < tail && atomicCAS(sd.head, head, head + 1) == head)
                return make_int4((int)(head % (unsigned long long)sd.cap), 0, -1, 1);
            ((volatile int*)mb)[3] = 0;
            __threadfence();
            atomicOr(word, bit);
            continue;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
}

static __device__ void fim_rer_accumulate(const NetDev& N, const double* __restrict__ c, const double* __restrict__ s,
                                   const unsigned long long* __restrict__ hist, const double* __restrict__ gradU_n,
                                   const double* __restrict__ gradV_n, const double* __restrict__ cprime,
                                   int n_cprime, double* fim_out, double* rer_out, int start, int stride);

// Outputs of a finished request, by the last block of its gang: the
// histogram normalised by T_s, the FIM and RER contracted over the post-burn
// histogram and divided by T_s - T_burn, the control block; then done.
static __device__ void serve_epilogue(const RunParams& P, const ServeSlot* slot, int* done) {
    __shared__ double s_c[8], s_s[4], s_cp[64];
    __shared__ int s_n, s_L;
    __shared__ double s_Tb;
    RunCtl* ctl = P.ctl;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) s_c[i] = slot->c[i];
        for (int i = 0; i < 4; ++i) s_s[i] = slot->s[i];
        s_n = slot->n_cprime < 8 ? slot->n_cprime : 8;
        s_L = slot->L;
        s_Tb = slot->T_burn;
        for (int i = 0; i < s_n * s_L; ++i) s_cp[i] = slot->cprime[i];
    }
    __syncwarp();
    double* out_hist = slot->out_hist;
    double* out_fim = slot->out_fim;
    double* out_rer = slot->out_rer;
    const double* gU = slot->gradU_n;
    const double* gV = slot->gradV_n;
    __syncthreads();
    const double Ts = (double)ldv(&ctl->Ts) * kQInv;
    const double scale = Ts > 0 ? 1.0 / Ts : 0.0;
    for (int b = threadIdx.x; b < P.net.nbins; b += blockDim.x) {
        const double a = (double)__ldcg(P.hist_pre + b) * kQInv, c = (double)__ldcg(P.hist_post + b) * kQInv;
        out_hist[b] = (a + c) * scale;
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) out_fim[i] = 0.0;
    for (int i = threadIdx.x; i < 8; i += blockDim.x) out_rer[i] = 0.0;
    __syncthreads();
    if (ldv(&ctl->status) == 0)
        fim_rer_accumulate(P.net, s_c, s_s, P.hist_post, gU, gV, s_cp, s_n, out_fim, out_rer, threadIdx.x,
                           blockDim.x);
    __syncthreads();
    const double span = Ts - s_Tb;
    if (span > 0.0) {
        if ((int)threadIdx.x < s_L * s_L) out_fim[threadIdx.x] /= span;
        if ((int)threadIdx.x < s_n) out_rer[threadIdx.x] /= span;
    }
    const unsigned long long* src = (const unsigned long long*)ctl;
    unsigned long long* dst = (unsigned long long*)slot->out_ctl;
    for (int i = threadIdx.x; i < (int)(sizeof(RunCtl) / 8); i += blockDim.x) dst[i] = ldv(src + i);
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0) st_release_sys(done, 1);
}

template <int FORM>
__global__ void PARREP_BOUNDS(FORM) parrep_serve_kernel(ServeDev sd) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockScratch red;
    __shared__ RunParams sP;
    __shared__ int4 s_cmd;
    for (;;) {
        if (threadIdx.x == 0) s_cmd = serve_next(sd);
        __syncwarp();
        __syncthreads();
        const int4 cmd = s_cmd;
        __syncthreads();
        if (cmd.w == 0) break;
        const ServeSlot* slot = sd.slots + cmd.x;
        const int* src = (const int*)&slot->P;
        int* dst = (int*)&sP;
        for (int w = threadIdx.x; w < (int)(sizeof(RunParams) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        if (cmd.w == 1) {
            // a new request: its leader clears the control block and the
            // histograms (no other block knows the request yet)
            unsigned long long* c = (unsigned long long*)sP.ctl;
            for (int i = threadIdx.x; i < (int)(sizeof(RunCtl) / 8); i += blockDim.x) c[i] = 0;
            for (int b = threadIdx.x; b < sP.net.nbins; b += blockDim.x) {
                sP.hist_pre[b] = 0;
                sP.hist_post[b] = 0;
            }
            __threadfence();
            __syncthreads();
        }
        const int join_gen = cmd.w == 2 ? cmd.z : -1;
        const bool last = run_any<FORM>(sP, cmd.y, smem, red, join_gen);
        if (last) {
            serve_epilogue(sP, slot, sd.done + cmd.x);
            if (threadIdx.x == 0) atomicAdd(sd.finished, 1ull);
        }
        __syncthreads();
    }
}

#if PARREP_PART == 0
// Zeroes the control block and the histograms of every instance of a batch
// (one block per instance).
__global__ void batch_reset_kernel(const RunParams* __restrict__ Ps, int n, BatchDev bd, int grid) {
    const RunParams& P = Ps[blockIdx.x];
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *bd.remaining = n;
        for (int w = threadIdx.x; w < (grid + 31) / 32; w += blockDim.x) bd.idle[w] = 0;
        for (int b = threadIdx.x; b < grid; b += blockDim.x) bd.mail[b] = make_int4(0, 0, 0, 0);
    }
    unsigned long long* c = (unsigned long long*)P.ctl;
    for (int i = threadIdx.x; i < (int)(sizeof(RunCtl) / 8); i += blockDim.x) c[i] = 0;
    for (int b = threadIdx.x; b < P.net.nbins; b += blockDim.x) {
        P.hist_pre[b] = 0;
        P.hist_post[b] = 0;
    }
}
#endif

#if PARREP_PART == 0
// Copies every instance's control block into one array for the host.
__global__ void batch_gather_kernel(const RunParams* __restrict__ Ps, int n, RunCtl* out) {
    const unsigned long long* c = (const unsigned long long*)Ps[blockIdx.x].ctl;
    unsigned long long* o = (unsigned long long*)(out + blockIdx.x);
    for (int i = threadIdx.x; i < (int)(sizeof(RunCtl) / 8); i += blockDim.x) o[i] = c[i];
}
#endif

// ---------------------------------------------------------------------------
// stand-alone dephasing (for tests and diagnostics)
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void dephase_kernel(RunParams P, int xt0, int xt1, int W, unsigned cycle, long long np, int* out,
                               int* status) {
    const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = (long long)r < (long long)P.R;
    int x0, x1;
    int st = dephase_warp<F32>(P.net, active, r, P.G, W, xt0, xt1, np, cycle, seed_key(P.seed), x0, x1);
    if (st && (threadIdx.x & 31) == 0) atomicCAS(status, 0, st);
    if (active) {
        out[2 * r] = x0;
        out[2 * r + 1] = x1;
    }
}

#if PARREP_PART == 0
// ---------------------------------------------------------------------------
// histogram normalisation, FIM and RER contractions (Sec. IV, Appendix A)
// ---------------------------------------------------------------------------
__global__ void hist_normalise_kernel(const unsigned long long* pre, const unsigned long long* post, int n,
                                      double scale, double* out_pre, double* out_post, double* out_norm) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const double a = (double)pre[b] * kQInv, c = (double)post[b] * kQInv;
        if (out_pre) out_pre[b] = a;
        if (out_post) out_post[b] = c;
        if (out_norm) out_norm[b] = (a + c) * scale;
    }
}
#endif

// Per bin: w = time in the bin; FIM += w sum_j lambda_j g_j g_j^T with
// g_j = grad_c log lambda_j; RER_k += w sum_j [lambda_j log(lambda_j/lambda'_j)
// - lambda_j + lambda'_j].
// The genetic switch (Sec. V.B): six channels, the eight parameters c = (a, b,
// gamma, k0min, k0max, k1min, k1max, D) taken independently.  With h =
// p^2/(p^2 + D^2), F = k0min + (k0max - k0min) h, G = k1max - (k1max - k1min) h:
//   log-derivatives of lambda = (a xi, gamma m, gamma b m, p, F (1 - xi), G xi):
//   d/da log l0 = 1/a; d/dgamma log l1 = 1/gamma; d/db log l2 = 1/b,
//   d/dgamma log l2 = 1/gamma; l3 has no parameter;
//   d/dk0min log l4 = (1 - h)/F, d/dk0max = h/F, d/dD = (k0max - k0min) h'/F;
//   d/dk1min log l5 = h/G, d/dk1max = (1 - h)/G, d/dD = -(k1max - k1min) h'/G,
//   h' = dh/dD = -2 p^2 D / (p^2 + D^2)^2.
// Per bin: FIM += w sum_j lambda_j g_j g_j^T; RER_k += w sum_j [lambda_j
// log(lambda_j/lambda'_j) - lambda_j + lambda'_j] with lambda' at c'_k.
static __device__ __forceinline__ void genetic_grad(const double* __restrict__ c, double p, double g[6][8]) {
    const double p2 = p * p, D2 = c[7] * c[7];
    const double h = p2 / (p2 + D2);
    const double dh = -2.0 * p2 * c[7] / ((p2 + D2) * (p2 + D2));
    const double F = c[3] + (c[4] - c[3]) * h, G = c[6] - (c[6] - c[5]) * h;
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int k = 0; k < 8; ++k) g[j][k] = 0.0;
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
}

static __device__ void fim_rer_genetic(const NetDev& N, const double* __restrict__ c,
                                       const unsigned long long* __restrict__ hist, const double* __restrict__ cprime,
                                       int n_cprime, double* fim_out, double* rer_out, int start, int stride) {
    constexpr int L = 8;
    double acc[L * L];
#pragma unroll
    for (int i = 0; i < L * L; ++i) acc[i] = 0.0;
    double racc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) racc[i] = 0.0;
    for (int b = start; b < N.nbins; b += stride) {
        const unsigned long long hq = __ldcg(hist + b);
        if (!hq) continue;
        const double w = (double)hq * kQInv;
        const int x0 = b / N.ystride, x1 = b % N.ystride;
        double lam[6];
        props6_d(N, x0, x1, lam);
        const double xi = (double)(x0 & 1), m = (double)(x0 >> 1), p = (double)x1;
        const double p2 = p * p;
        double g[6][L];
        genetic_grad(c, p, g);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (lam[j] == 0.0) continue;
#pragma unroll
            for (int a = 0; a < L; ++a)
#pragma unroll
                for (int bb = 0; bb < L; ++bb) acc[a * L + bb] += w * lam[j] * g[j][a] * g[j][bb];
        }
        for (int k = 0; k < n_cprime && k < 8; ++k) {
            const double* cp = cprime + k * L;
            const double D2p = cp[7] * cp[7];
            const double hp = p2 / (p2 + D2p);
            const double Fp = cp[3] + (cp[4] - cp[3]) * hp, Gp = cp[6] - (cp[6] - cp[5]) * hp;
            const double lp[6] = {cp[0] * xi, cp[2] * m, (cp[2] * cp[1]) * m, p, Fp * (1.0 - xi), Gp * xi};
            double hsum = 0.0;
            for (int j = 0; j < 6; ++j) {
                double t = lp[j] - lam[j];
                if (lam[j] > 0.0) t += lam[j] * log(lam[j] / lp[j]);
                hsum += t;
            }
            racc[k] += w * hsum;
        }
    }
    for (int i = 0; i < L * L; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(fim_out + i, v);
    }
    for (int k = 0; k < n_cprime && k < 8; ++k) {
        double v = racc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(rer_out + k, v);
    }
}

static __device__ void fim_rer_accumulate(const NetDev& N, const double* __restrict__ c, const double* __restrict__ s,
                                   const unsigned long long* __restrict__ hist, const double* __restrict__ gradU_n,
                                   const double* __restrict__ gradV_n, const double* __restrict__ cprime,
                                   int n_cprime, double* fim_out, double* rer_out, int start, int stride) {
    if (N.kind == PARREP_GENETIC) {
        fim_rer_genetic(N, c, hist, cprime, n_cprime, fim_out, rer_out, start, stride);
        return;
    }
    const int L = N.kind == PARREP_SCHLOGL ? 4 : 6;
    double acc[36];
#pragma unroll
    for (int i = 0; i < 36; ++i) acc[i] = 0.0;
    double racc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) racc[i] = 0.0;
    for (int b = start; b < N.nbins; b += stride) {
        const unsigned long long hq = __ldcg(hist + b);
        if (!hq) continue;
        const double w = (double)hq * kQInv;
        const int x0 = b / N.ystride, x1 = b % N.ystride;
        double lam[4];
        props_d(N, x0, x1, lam[0], lam[1], lam[2], lam[3]);
        double g[4][6];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 6; ++k) g[j][k] = 0.0;
        if (N.kind == PARREP_SCHLOGL) {
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j][j] = 1.0 / c[j];
        } else {
            g[0][0] = 1.0 / c[0];
            g[0][1] = gradU_n[x1];
            g[1][3] = 1.0 / c[3];
            g[1][4] = gradV_n[x0];
            g[2][2] = 1.0 / c[2];
            g[3][5] = 1.0 / c[5];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (lam[j] == 0.0) continue;
            for (int a = 0; a < L; ++a)
                for (int bb = 0; bb < L; ++bb) acc[a * L + bb] += w * lam[j] * g[j][a] * g[j][bb];
        }
        for (int k = 0; k < n_cprime && k < 8; ++k) {
            const double* cp = cprime + k * L;
            double lp[4];
            if (N.kind == PARREP_SCHLOGL) {
                const double xd = (double)x0;
                const double h1 = xd * (xd - 1.0), h2 = h1 * (xd - 2.0);
                lp[0] = (cp[0] * s[0]) * h1;
                lp[1] = (cp[1] * s[1]) * h2;
                lp[2] = (cp[2] * s[2]);
                lp[3] = (cp[3] * s[3]) * xd;
            } else {
                lp[0] = cp[0] / (1.0 + pow((double)x1, cp[1]));
                lp[1] = cp[3] / (1.0 + pow((double)x0, cp[4]));
                lp[2] = cp[2] * (double)x0;
                lp[3] = cp[5] * (double)x1;
            }
            double h = 0.0;
            for (int j = 0; j < 4; ++j) {
                double t = lp[j] - lam[j];
                if (lam[j] > 0.0) t += lam[j] * log(lam[j] / lp[j]);
                h += t;
            }
            racc[k] += w * h;
        }
    }
    for (int i = 0; i < L * L; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(fim_out + i, v);
    }
    for (int k = 0; k < n_cprime && k < 8; ++k) {
        double v = racc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(rer_out + k, v);
    }
}

#if PARREP_PART == 0
__global__ void fim_rer_kernel(NetDev N, const double* __restrict__ c, const double* __restrict__ s,
                               const unsigned long long* __restrict__ hist, const double* __restrict__ gradU_n,
                               const double* __restrict__ gradV_n, const double* __restrict__ cprime, int n_cprime,
                               double* fim_out, double* rer_out) {
    fim_rer_accumulate(N, c, s, hist, gradU_n, gradV_n, cprime, n_cprime, fim_out, rer_out,
                       blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}
#endif

// ---------------------------------------------------------------------------
// stationary UQ over independent runs (Sec. IV.B)
// ---------------------------------------------------------------------------
constexpr int kUqThreads = 256;

// Sum of v over the block in a fixed order: an xor butterfly inside each warp
// (both partners add the same two values, so every lane holds the same
// bits), then the warps' sums in warp order by thread 0.  red holds one slot
// per warp; the result is valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

#if PARREP_PART == 0
// One block per sample k: Y[k] = sum_b f[b] * time(b) over the post-burn
// sums, and Z[k] = the FIM time average (the parrep_fim contraction: per bin
// w sum_j lambda_j g_j g_j^T with g_j = grad_c log lambda_j, over the window).
__global__ void __launch_bounds__(kUqThreads) uq_sample_kernel(const UqSample* __restrict__ smp,
                                                                const double* __restrict__ f, int L, double window,
                                                                double* __restrict__ Y, double* __restrict__ Z) {
    __shared__ double red[kUqThreads / 32];
    const UqSample& S = smp[blockIdx.x];
    const NetDev& N = S.net;
    double y = 0.0;
    double acc[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.0;
    double ic[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) ic[i] = i < L ? 1.0 / S.c[i] : 0.0;
    const bool gen = N.kind == PARREP_GENETIC;
    const int nch = gen ? 6 : 4;
    for (int b = threadIdx.x; b < N.nbins; b += blockDim.x) {
        const unsigned long long hq = __ldcg(S.hist + b);
        if (!hq) continue;
        const double w = (double)hq * kQInv;
        y += f[b] * w;
        const int x0 = b / N.ystride, x1 = b % N.ystride;
        double lam[6];
        double g[6][8];
        if (gen) {
            props6_d(N, x0, x1, lam);
            genetic_grad(S.c, (double)x1, g);
        } else {
            props_d(N, x0, x1, lam[0], lam[1], lam[2], lam[3]);
            lam[4] = lam[5] = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j)
#pragma unroll
                for (int k = 0; k < 8; ++k) g[j][k] = 0.0;
            if (N.kind == PARREP_SCHLOGL) {
#pragma unroll
                for (int j = 0; j < 4; ++j) g[j][j] = ic[j];
            } else {
                g[0][0] = ic[0];
                g[0][1] = S.gradU_n[x1];
                g[1][3] = ic[3];
                g[1][4] = S.gradV_n[x0];
                g[2][2] = ic[2];
                g[3][5] = ic[5];
            }
        }
        for (int j = 0; j < nch; ++j) {
            if (lam[j] == 0.0) continue;
            for (int a = 0; a < L; ++a)
                for (int bb = 0; bb < L; ++bb) acc[a * L + bb] += w * lam[j] * g[j][a] * g[j][bb];
        }
    }
    const double yt = block_sum_fixed(y, red);
    if (threadIdx.x == 0) Y[blockIdx.x] = yt;
    for (int i = 0; i < L * L; ++i) {
        const double t = block_sum_fixed(acc[i], red);
        if (threadIdx.x == 0) Z[(size_t)blockIdx.x * 64 + i] = t / window;
    }
}
#endif

#if PARREP_PART == 0
// One block: moments of Y (two passes), mean and 95% half width of each FIM
// entry over the samples, and the bounds sqrt(tau) sqrt(v^T I v) -- each sum
// in sample order.
__global__ void uq_reduce_kernel(int n, int L, const double* __restrict__ Y, const double* __restrict__ Z,
                                 double window, const double* __restrict__ dirs, int n_dirs, UqOut* out,
                                 double* dir_bounds) {
    __shared__ double sh_tau;
    __shared__ double sh_fim[64];
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int k = threadIdx.x; k < n; k += 32) s += Y[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double ybar = s / (double)n;
        double v = 0.0;
        for (int k = threadIdx.x; k < n; k += 32) {
            const double d = Y[k] - ybar;
            v += d * d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) {
            const double tau = v / (window * (double)(n - 1));
            out->iaf = tau;
            out->mean_f = ybar / window;
            sh_tau = tau;
        }
    }
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        double m = 0.0, hw = 0.0;
        if (t < L * L) {
            for (int k = 0; k < n; ++k) m += Z[(size_t)k * 64 + t];
            m /= (double)n;
            double v = 0.0;
            for (int k = 0; k < n; ++k) {
                const double d = Z[(size_t)k * 64 + t] - m;
                v += d * d;
            }
            hw = 1.96 * sqrt(v / (double)(n - 1)) / sqrt((double)n);
        }
        out->fim[t] = m;
        out->half[t] = hw;
        sh_fim[t] = m;
    }
    __syncthreads();
    const double rt = sqrt(sh_tau);
    for (int j = threadIdx.x; j < 8; j += blockDim.x) out->bound[j] = j < L ? rt * sqrt(fmax(sh_fim[j * L + j], 0.0)) : 0.0;
    for (int d = threadIdx.x; d < n_dirs; d += blockDim.x) {
        const double* v = dirs + (size_t)d * L;
        double q = 0.0;
        for (int a = 0; a < L; ++a) {
            double r = 0.0;
            for (int b = 0; b < L; ++b) r += sh_fim[a * L + b] * v[b];
            q += v[a] * r;
        }
        dir_bounds[d] = rt * sqrt(fmax(q, 0.0));
    }
}
#endif

// ---------------------------------------------------------------------------
// plain SSA: one thread per independent trajectory
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void ssa_kernel(NetDev N, long long n_traj, int x00, int x01, unsigned long long q_Tend,
                           unsigned long long seed, unsigned long long* hist, unsigned long long* events,
                           int* status) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long ev = 0;
    if (t < n_traj) {
        const uint2 key = seed_key(seed);
        int x0 = x00, x1 = x01;
        unsigned long long T = 0, step = 0;
        while (T < q_Tend) {
            const unsigned long long cs = F32 ? step >> 1 : step;
            uint4 w = philox10(make_uint4((unsigned)t, (unsigned)cs, (unsigned)(cs >> 32), kTagSSA), key);
            if (F32 && (step & 1)) w = make_uint4(w.z, w.w, 0u, 0u);
            unsigned long long q = 0;
            const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
            const unsigned long long rem = q_Tend - T;
            const int b = x0 * N.ystride + x1;
            if (q >= rem) {
                atomicAdd(hist + b, rem);
                break;
            }
            atomicAdd(hist + b, q);
            T += q;
            apply(N, J, x0, x1);
            ++ev;
            ++step;
            if (out_of_range(N, x0, x1)) {
                atomicCAS(status, 0, PARREP_ERANGE);
                break;
            }
        }
    }
    ev = warp_sum(ev);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd(events, ev);
}

// Plain SSA with a per-jump record, for trajectory parity tests: the same
// counters and arithmetic as ssa_kernel; trajectory t stops at T_end or after
// max_steps jumps and writes, per jump, the channel, the state after the jump
// and the fixed-point holding time, then its jump count and final state.
template <bool F32>
__global__ void ssa_trace_kernel(NetDev N, long long n_traj, int x00, int x01, unsigned long long q_Tend,
                                 unsigned long long seed, long long max_steps, int* J_out, int2* x_out,
                                 unsigned long long* q_out, long long* n_out, int2* xf_out, int* status) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_traj) return;
    const uint2 key = seed_key(seed);
    int x0 = x00, x1 = x01;
    unsigned long long T = 0, step = 0;
    const size_t base = (size_t)t * (size_t)max_steps;
    while (T < q_Tend && (long long)step < max_steps) {
        const unsigned long long cs = F32 ? step >> 1 : step;
        uint4 w = philox10(make_uint4((unsigned)t, (unsigned)cs, (unsigned)(cs >> 32), kTagSSA), key);
        if (F32 && (step & 1)) w = make_uint4(w.z, w.w, 0u, 0u);
        unsigned long long q = 0;
        const int J = ssa_draw<F32, true>(N, x0, x1, w, q);
        if (q >= q_Tend - T) break;  // the jump falls after T_end
        T += q;
        apply(N, J, x0, x1);
        J_out[base + step] = J;
        x_out[base + step] = make_int2(x0, x1);
        q_out[base + step] = q;
        ++step;
        if (out_of_range(N, x0, x1)) {
            atomicCAS(status, 0, PARREP_ERANGE);
            break;
        }
    }
    n_out[t] = (long long)step;
    xf_out[t] = make_int2(x0, x1);
}

#if PARREP_PART == 0
__global__ void philox_kernel(const uint4* ctr, const uint2* key, long long n, uint4* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox10(ctr[i], key[i]);
}
#endif

// ---------------------------------------------------------------------------
// launchers (one precision and one kernel family per part)
// ---------------------------------------------------------------------------
// per form (0 = binary64, 1 = binary32 staged, 2 = binary32 direct)
int kernel_attrs_form(int form, int kind, int* max_blocks_per_sm, int smem_bytes, int threads);
cudaError_t launch_run_form(const RunParams& p, int grid, int threads, int smem_bytes, cudaStream_t st);
int batch_attrs_form(int form, int* max_blocks_per_sm, int smem_bytes, int threads);
cudaError_t launch_batch_form(int form, const cudaLaunchConfig_t& cfg, const RunParams* d_params, const int* d_off,
                              const int2* d_items, BatchDev bd);
int serve_attrs_form(int form, int* max_blocks_per_sm, int smem_bytes, int threads);
cudaError_t launch_serve_form(int form, const ServeDev& sd, int grid, int threads, int smem_bytes, cudaStream_t st);

template <typename K>
static int attrs_of(K kernel, int* max_blocks_per_sm, int smem_bytes, int threads) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, kernel, threads, smem_bytes);
    return (int)e;
}

// parts 1-3: the run kernels, parts 4-6: the batch kernels, parts 7-9: the
// serve kernels, each in binary64, binary32 staged and binary32 direct form
#if PARREP_PART >= 1 && PARREP_PART <= 9
constexpr int kPartForm = (PARREP_PART - 1) % 3;
#endif

// parts 10 and 11: the batch and serve kernels in the mixed binary32 form
#if PARREP_PART == 10
int batch_attrs_f32m(int* m, int s, int t) { return attrs_of(parrep_batch_kernel<kFormF32Mixed>, m, s, t); }
cudaError_t batch_launch_f32m(const cudaLaunchConfig_t& c, const RunParams* p, const int* o, const int2* i, BatchDev b) {
    return cudaLaunchKernelEx(&c, parrep_batch_kernel<kFormF32Mixed>, p, o, i, b);
}
#endif
#if PARREP_PART == 11
int serve_attrs_f32m(int* m, int s, int t) { return attrs_of(parrep_serve_kernel<kFormF32Mixed>, m, s, t); }
cudaError_t serve_launch_f32m(const ServeDev& d, int g, int t, int s, cudaStream_t st) {
    parrep_serve_kernel<kFormF32Mixed><<<g, t, s, st>>>(d);
    return cudaGetLastError();
}
#endif

#if PARREP_PART >= 1 && PARREP_PART <= 3
// The genetic switch runs in the two-species instantiation (its channels are
// chosen by N.kind inside).
static int run_attrs_here(int kind, int* max_blocks_per_sm, int smem_bytes, int threads) {
    return kind == PARREP_SCHLOGL
               ? attrs_of(parrep_run_kernel<kPartForm, PARREP_SCHLOGL>, max_blocks_per_sm, smem_bytes, threads)
               : attrs_of(parrep_run_kernel<kPartForm, PARREP_TOGGLE>, max_blocks_per_sm, smem_bytes, threads);
}
static cudaError_t run_launch_here(const RunParams& p, int grid, int threads, int smem_bytes, cudaStream_t st) {
    void* args[] = {(void*)&p};
    void* fn = p.net.kind == PARREP_SCHLOGL ? (void*)parrep_run_kernel<kPartForm, PARREP_SCHLOGL>
                                            : (void*)parrep_run_kernel<kPartForm, PARREP_TOGGLE>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, (size_t)smem_bytes, st);
}
#if PARREP_PART == 1
int run_attrs_f64(int kind, int* m, int s, int t) { return run_attrs_here(kind, m, s, t); }
cudaError_t run_launch_f64(const RunParams& p, int g, int t, int s, cudaStream_t st) { return run_launch_here(p, g, t, s, st); }
#elif PARREP_PART == 2
int run_attrs_f32s(int kind, int* m, int s, int t) { return run_attrs_here(kind, m, s, t); }
cudaError_t run_launch_f32s(const RunParams& p, int g, int t, int s, cudaStream_t st) { return run_launch_here(p, g, t, s, st); }
#else
int run_attrs_f32d(int kind, int* m, int s, int t) { return run_attrs_here(kind, m, s, t); }
cudaError_t run_launch_f32d(const RunParams& p, int g, int t, int s, cudaStream_t st) { return run_launch_here(p, g, t, s, st); }
#endif
#endif

#if PARREP_PART >= 4 && PARREP_PART <= 6
static int batch_attrs_here(int* max_blocks_per_sm, int smem_bytes, int threads) {
    return attrs_of(parrep_batch_kernel<kPartForm>, max_blocks_per_sm, smem_bytes, threads);
}
static cudaError_t batch_launch_here(const cudaLaunchConfig_t& cfg, const RunParams* d_params, const int* d_off,
                                     const int2* d_items, BatchDev bd) {
    return cudaLaunchKernelEx(&cfg, parrep_batch_kernel<kPartForm>, d_params, d_off, d_items, bd);
}
#if PARREP_PART == 4
int batch_attrs_f64(int* m, int s, int t) { return batch_attrs_here(m, s, t); }
cudaError_t batch_launch_f64(const cudaLaunchConfig_t& c, const RunParams* p, const int* o, const int2* i, BatchDev b) {
    return batch_launch_here(c, p, o, i, b);
}
#elif PARREP_PART == 5
int batch_attrs_f32s(int* m, int s, int t) { return batch_attrs_here(m, s, t); }
cudaError_t batch_launch_f32s(const cudaLaunchConfig_t& c, const RunParams* p, const int* o, const int2* i, BatchDev b) {
    return batch_launch_here(c, p, o, i, b);
}
#else
int batch_attrs_f32d(int* m, int s, int t) { return batch_attrs_here(m, s, t); }
cudaError_t batch_launch_f32d(const cudaLaunchConfig_t& c, const RunParams* p, const int* o, const int2* i, BatchDev b) {
    return batch_launch_here(c, p, o, i, b);
}
#endif
#endif

#if PARREP_PART >= 7 && PARREP_PART <= 9
static int serve_attrs_here(int* max_blocks_per_sm, int smem_bytes, int threads) {
    return attrs_of(parrep_serve_kernel<kPartForm>, max_blocks_per_sm, smem_bytes, threads);
}
static cudaError_t serve_launch_here(const ServeDev& sd, int grid, int threads, int smem_bytes, cudaStream_t st) {
    parrep_serve_kernel<kPartForm><<<grid, threads, smem_bytes, st>>>(sd);
    return cudaGetLastError();
}
#if PARREP_PART == 7
int serve_attrs_f64(int* m, int s, int t) { return serve_attrs_here(m, s, t); }
cudaError_t serve_launch_f64(const ServeDev& d, int g, int t, int s, cudaStream_t st) { return serve_launch_here(d, g, t, s, st); }
#elif PARREP_PART == 8
int serve_attrs_f32s(int* m, int s, int t) { return serve_attrs_here(m, s, t); }
cudaError_t serve_launch_f32s(const ServeDev& d, int g, int t, int s, cudaStream_t st) { return serve_launch_here(d, g, t, s, st); }
#else
int serve_attrs_f32d(int* m, int s, int t) { return serve_attrs_here(m, s, t); }
cudaError_t serve_launch_f32d(const ServeDev& d, int g, int t, int s, cudaStream_t st) { return serve_launch_here(d, g, t, s, st); }
#endif
#endif

#if PARREP_PART == 0
int run_attrs_f64(int, int*, int, int);
int run_attrs_f32s(int, int*, int, int);
int run_attrs_f32d(int, int*, int, int);
cudaError_t run_launch_f64(const RunParams&, int, int, int, cudaStream_t);
cudaError_t run_launch_f32s(const RunParams&, int, int, int, cudaStream_t);
cudaError_t run_launch_f32d(const RunParams&, int, int, int, cudaStream_t);
int batch_attrs_f64(int*, int, int);
int batch_attrs_f32s(int*, int, int);
int batch_attrs_f32d(int*, int, int);
cudaError_t batch_launch_f64(const cudaLaunchConfig_t&, const RunParams*, const int*, const int2*, BatchDev);
cudaError_t batch_launch_f32s(const cudaLaunchConfig_t&, const RunParams*, const int*, const int2*, BatchDev);
cudaError_t batch_launch_f32d(const cudaLaunchConfig_t&, const RunParams*, const int*, const int2*, BatchDev);
int serve_attrs_f64(int*, int, int);
int serve_attrs_f32s(int*, int, int);
int serve_attrs_f32d(int*, int, int);
cudaError_t serve_launch_f64(const ServeDev&, int, int, int, cudaStream_t);
cudaError_t serve_launch_f32s(const ServeDev&, int, int, int, cudaStream_t);
cudaError_t serve_launch_f32d(const ServeDev&, int, int, int, cudaStream_t);
int batch_attrs_f32m(int*, int, int);
cudaError_t batch_launch_f32m(const cudaLaunchConfig_t&, const RunParams*, const int*, const int2*, BatchDev);
int serve_attrs_f32m(int*, int, int);
cudaError_t serve_launch_f32m(const ServeDev&, int, int, int, cudaStream_t);

int kernel_attrs_form(int form, int kind, int* m, int s, int t) {
    return form == kFormF32Direct ? run_attrs_f32d(kind, m, s, t)
           : form == kFormF32Staged ? run_attrs_f32s(kind, m, s, t)
                                    : run_attrs_f64(kind, m, s, t);
}

cudaError_t launch_run(const RunParams& p, int grid, int threads, int smem_bytes, cudaStream_t st) {
    return p.form == kFormF32Direct ? run_launch_f32d(p, grid, threads, smem_bytes, st)
           : p.form == kFormF32Staged ? run_launch_f32s(p, grid, threads, smem_bytes, st)
                                      : run_launch_f64(p, grid, threads, smem_bytes, st);
}

int batch_attrs_form(int form, int* m, int s, int t) {
    return form == kFormF32Mixed    ? batch_attrs_f32m(m, s, t)
           : form == kFormF32Direct ? batch_attrs_f32d(m, s, t)
           : form == kFormF32Staged ? batch_attrs_f32s(m, s, t)
                                    : batch_attrs_f64(m, s, t);
}

cudaError_t launch_batch(int form, const RunParams* d_params, int n, const int* d_off, const int2* d_items,
                         BatchDev bd, int grid, int threads, int smem_bytes, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    batch_reset_kernel<<<n, 256, 0, st>>>(d_params, n, bd, grid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = (size_t)smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return form == kFormF32Mixed    ? batch_launch_f32m(cfg, d_params, d_off, d_items, bd)
           : form == kFormF32Direct ? batch_launch_f32d(cfg, d_params, d_off, d_items, bd)
           : form == kFormF32Staged ? batch_launch_f32s(cfg, d_params, d_off, d_items, bd)
                                    : batch_launch_f64(cfg, d_params, d_off, d_items, bd);
}

cudaError_t launch_batch_gather(const RunParams* d_params, int n, RunCtl* out, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    batch_gather_kernel<<<n, 64, 0, st>>>(d_params, n, out);
    return cudaGetLastError();
}

int serve_attrs_form(int form, int* m, int s, int t) {
    return form == kFormF32Mixed    ? serve_attrs_f32m(m, s, t)
           : form == kFormF32Direct ? serve_attrs_f32d(m, s, t)
           : form == kFormF32Staged ? serve_attrs_f32s(m, s, t)
                                    : serve_attrs_f64(m, s, t);
}

cudaError_t launch_serve(int form, const ServeDev& sd, int grid, int threads, int smem_bytes, cudaStream_t st) {
    return form == kFormF32Mixed    ? serve_launch_f32m(sd, grid, threads, smem_bytes, st)
           : form == kFormF32Direct ? serve_launch_f32d(sd, grid, threads, smem_bytes, st)
           : form == kFormF32Staged ? serve_launch_f32s(sd, grid, threads, smem_bytes, st)
                                    : serve_launch_f64(sd, grid, threads, smem_bytes, st);
}

cudaError_t launch_dephase(const RunParams& p, int xt0, int xt1, int W, unsigned cycle, long long np,
                           int* out_states, int grid, int threads, cudaStream_t st) {
    int* status = &p.ctl->status;
    if (p.prec == PARREP_FP32)
        dephase_kernel<true><<<grid, threads, 0, st>>>(p, xt0, xt1, W, cycle, np, out_states, status);
    else
        dephase_kernel<false><<<grid, threads, 0, st>>>(p, xt0, xt1, W, cycle, np, out_states, status);
    return cudaGetLastError();
}

cudaError_t launch_hist_normalise(const unsigned long long* pre, const unsigned long long* post, int n, double scale,
                                  double* out_pre, double* out_post, double* out_norm, cudaStream_t st) {
    int blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    hist_normalise_kernel<<<blocks, 256, 0, st>>>(pre, post, n, scale, out_pre, out_post, out_norm);
    return cudaGetLastError();
}

cudaError_t launch_fim_rer(const NetDev& net, const double* c, const double* s, const unsigned long long* hist,
                           const double* gradU_n, const double* gradV_n, const double* cprime, int n_cprime,
                           double* fim_out, double* rer_out, cudaStream_t st) {
    int blocks = (net.nbins + 127) / 128;
    if (blocks > 304) blocks = 304;
    if (blocks < 1) blocks = 1;
    fim_rer_kernel<<<blocks, 128, 0, st>>>(net, c, s, hist, gradU_n, gradV_n, cprime, n_cprime, fim_out, rer_out);
    return cudaGetLastError();
}

cudaError_t launch_uq(const UqSample* samples, int n, int L, const double* f, double window, const double* dirs,
                      int n_dirs, double* Y, double* Z, UqOut* out, double* dir_bounds, cudaStream_t st) {
    uq_sample_kernel<<<n, kUqThreads, 0, st>>>(samples, f, L, window, Y, Z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uq_reduce_kernel<<<1, 64, 0, st>>>(n, L, Y, Z, window, dirs, n_dirs, out, dir_bounds);
    return cudaGetLastError();
}

cudaError_t launch_ssa(const NetDev& net, int prec, long long n_traj, int x0, int x1, unsigned long long q_Tend,
                       unsigned long long seed, unsigned long long* hist, unsigned long long* events, int* status,
                       cudaStream_t st) {
    const int threads = 128;
    const long long blocks = (n_traj + threads - 1) / threads;
    if (prec == PARREP_FP32)
        ssa_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(net, n_traj, x0, x1, q_Tend, seed, hist, events,
                                                               status);
    else
        ssa_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(net, n_traj, x0, x1, q_Tend, seed, hist, events,
                                                                status);
    return cudaGetLastError();
}

cudaError_t launch_ssa_trace(const NetDev& net, int prec, long long n_traj, int x0, int x1,
                             unsigned long long q_Tend, unsigned long long seed, long long max_steps, int* J,
                             int2* xs, unsigned long long* q, long long* n_out, int2* xf, int* status,
                             cudaStream_t st) {
    const int threads = 128;
    const long long blocks = (n_traj + threads - 1) / threads;
    if (prec == PARREP_FP32)
        ssa_trace_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(net, n_traj, x0, x1, q_Tend, seed, max_steps, J,
                                                                     xs, q, n_out, xf, status);
    else
        ssa_trace_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(net, n_traj, x0, x1, q_Tend, seed, max_steps,
                                                                      J, xs, q, n_out, xf, status);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, long long n, uint32_t* out, cudaStream_t st) {
    const int threads = 128;
    const long long blocks = (n + threads - 1) / threads;
    philox_kernel<<<(unsigned)blocks, threads, 0, st>>>((const uint4*)ctr, (const uint2*)key, n, (uint4*)out);
    return cudaGetLastError();
}

#endif  // PARREP_PART == 0

}  // namespace parrep
