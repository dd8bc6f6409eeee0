"""Python face of the C ABI (include/parrep.h): the same entry points, with
numpy / torch buffers marshalled to plain pointers.  Every step of the method
runs in the CUDA library; this module only converts arguments and results.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


class ParRepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{L.ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, h=None):
    if rc != L.PARREP_OK:
        lib = L.load()
        msg = lib.parrep_last_error(h)
        raise ParRepError(rc, msg.decode() if msg else "")
    return rc


def make_network(spec: dict, x0=None, x0_uniform_hi: int = 0) -> L.parrep_network:
    """parrep_network from a network spec dict (see configs)."""
    n = L.parrep_network()
    n.kind = {"schlogl": L.PARREP_SCHLOGL, "toggle": L.PARREP_TOGGLE, "genetic": L.PARREP_GENETIC}[spec["kind"]]
    n.n_species = 1 if n.kind == L.PARREP_SCHLOGL else 2
    for i, v in enumerate(spec["c"]):
        n.c[i] = float(v)
    for i, v in enumerate(spec.get("s", [1.0] * 4)):
        n.s[i] = float(v)
    hm = spec["hist_max"]
    hm = [hm] if np.isscalar(hm) else list(hm)
    n.hist_max[0] = int(hm[0])
    n.hist_max[1] = int(hm[1]) if len(hm) > 1 else 0
    x0 = [0, 0] if x0 is None else ([x0] if np.isscalar(x0) else list(x0))
    n.x0[0] = int(x0[0])
    n.x0[1] = int(x0[1]) if len(x0) > 1 else 0
    n.x0_uniform_hi = int(x0_uniform_hi)
    return n


def make_regions(spec: dict) -> L.parrep_regions:
    r = L.parrep_regions()
    regs = spec["regions"]
    r.n = len(regs)
    for i, (a, b) in enumerate(regs):
        a = list(a) + [0] * (2 - len(a))
        r.a[i][0] = int(a[0])
        r.a[i][1] = int(a[1])
        r.b[i] = int(b)
    return r


def _buf(x):
    """Pointer of a numpy array or a torch tensor (host or CUDA)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return C.c_void_p(x.data_ptr())
    raise TypeError("expected a numpy array or a torch tensor")


class ParRep:
    """Handle of parrep_create / parrep_destroy with the other entry points as
    methods of the same names (without the prefix)."""

    def __init__(self, spec: dict, n_replicas: int, t_corr: float, t_phase: float, *, x0=None,
                 x0_uniform_hi: int = 0, thresh: str = "time", precision: str = "f64", fv_group: int = 32,
                 T_burn: float = 0.0, block_threads: int = 0, chunk_steps: int = 0, stream=None,
                 wait_timeout_s: float = 10.0, debug_stall_barrier: int = -1, serial_stages: int = 0,
                 max_blocks: int = 0, f32_layout: str = "auto"):
        self._lib = L.load()
        self.spec = spec
        self.L = {"schlogl": 4, "toggle": 6, "genetic": 8}[spec["kind"]]
        self._net = make_network(spec, x0, x0_uniform_hi)
        self._reg = make_regions(spec)
        h = C.c_void_p()
        _check(self._lib.parrep_create(C.byref(self._net), int(n_replicas), C.byref(self._reg), float(t_corr),
                                       float(t_phase), C.byref(h)))
        self.h = h
        self.n_replicas = int(n_replicas)
        self.set_options(thresh=thresh, precision=precision, fv_group=fv_group, T_burn=T_burn,
                         block_threads=block_threads, chunk_steps=chunk_steps, stream=stream,
                         wait_timeout_s=wait_timeout_s, debug_stall_barrier=debug_stall_barrier,
                         serial_stages=serial_stages, max_blocks=max_blocks, f32_layout=f32_layout)

    def set_options(self, *, thresh="time", precision="f64", fv_group=32, T_burn=0.0, block_threads=0,
                    chunk_steps=0, stream=None, wait_timeout_s=10.0, debug_stall_barrier=-1, serial_stages=0,
                    max_blocks=0, f32_layout="auto"):
        o = L.parrep_options()
        self._lib.parrep_default_options(C.byref(o))
        o.thresh_mode = L.PARREP_THRESH_STEPS if thresh == "steps" else L.PARREP_THRESH_TIME
        o.precision = L.PARREP_FP32 if precision == "f32" else L.PARREP_FP64
        o.fv_group = int(fv_group)
        o.block_threads = int(block_threads)
        o.chunk_steps = int(chunk_steps)
        o.T_burn = float(T_burn)
        o.wait_timeout_s = float(wait_timeout_s)
        o.debug_stall_barrier = int(debug_stall_barrier)
        o.serial_stages = int(serial_stages)
        o.max_blocks = int(max_blocks)
        o.f32_layout = L.LAYOUTS[f32_layout]
        if stream is not None:
            o.stream = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        _check(self._lib.parrep_set_options(self.h, C.byref(o)), self.h)
        self._opt = o

    # -- run --
    def run(self, T_end: float, seed: int):
        _check(self._lib.parrep_run(self.h, float(T_end), int(seed) & 0xFFFFFFFFFFFFFFFF), self.h)
        return self.stats()

    def run_status(self, T_end: float, seed: int) -> int:
        """parrep_run returning the status code instead of raising."""
        return self._lib.parrep_run(self.h, float(T_end), int(seed) & 0xFFFFFFFFFFFFFFFF)

    @property
    def n_bins(self) -> int:
        return int(self._lib.parrep_n_bins(self.h))

    # -- outputs --
    def histogram(self, out=None):
        if out is None:
            out = np.zeros(self.n_bins)
        _check(self._lib.parrep_histogram(self.h, _buf(out), self.n_bins), self.h)
        return out

    def histogram_raw(self):
        pre = np.zeros(self.n_bins)
        post = np.zeros(self.n_bins)
        _check(self._lib.parrep_histogram_raw(self.h, _buf(pre), _buf(post), self.n_bins), self.h)
        return pre, post

    def fim(self, out=None):
        if out is None:
            out = np.zeros((self.L, self.L))
        _check(self._lib.parrep_fim(self.h, _buf(out), self.L * self.L), self.h)
        return out

    def rer(self, c_prime):
        cp = np.ascontiguousarray(c_prime, dtype=np.float64).reshape(-1, self.L)
        out = np.zeros(len(cp))
        _check(self._lib.parrep_rer(self.h, _buf(cp), len(cp), _buf(out)), self.h)
        return out

    def stats(self) -> dict:
        s = L.parrep_stats()
        _check(self._lib.parrep_stats_get(self.h, C.byref(s)), self.h)
        return _stats_dict(s)

    def cycle_log(self, cap: int = 65536):
        buf = (L.parrep_cycle * max(cap, 1))()
        n = C.c_int64(0)
        _check(self._lib.parrep_cycle_log(self.h, buf, cap, C.byref(n)), self.h)
        m = min(n.value, cap)
        return [dict(cycle=buf[i].cycle, W=buf[i].W, ended=buf[i].ended, decorr_steps=buf[i].decorr_steps,
                     dephase_steps=buf[i].dephase_steps, n_star=buf[i].n_star, k=buf[i].k,
                     x_tilde=(buf[i].x_tilde[0], buf[i].x_tilde[1]), T_s=buf[i].T_s) for i in range(m)]

    def dephase(self, x_tilde, W: int, cycle: int, seed: int):
        xt = (C.c_int32 * 2)(*(list(x_tilde) + [0] * (2 - len(x_tilde))))
        out = np.zeros((self.n_replicas, 2), dtype=np.int32)
        _check(self._lib.parrep_dephase(self.h, xt, int(W), int(cycle), int(seed), _buf(out)), self.h)
        return out

    def close(self):
        if getattr(self, "h", None):
            self._lib.parrep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class ParRepBatch:
    """parrep_batch_create / run / destroy over ParRep handles.  After run()
    every handle holds its own results (read them with its methods)."""

    def __init__(self, instances, *, block_threads: int = 0, replicas_per_block: int = 0, autotune: bool = True,
                 use_graph: bool = True, tune_fraction: float = 0.05, wait_timeout_s: float = 10.0, stream=None,
                 f32_layout: str = "auto"):
        self._lib = L.load()
        self.instances = list(instances)
        o = L.parrep_batch_options()
        self._lib.parrep_batch_default_options(C.byref(o))
        o.block_threads = int(block_threads)
        o.replicas_per_block = int(replicas_per_block)
        o.autotune = 1 if autotune else 0
        o.use_graph = 1 if use_graph else 0
        o.f32_layout = L.LAYOUTS[f32_layout]
        o.tune_fraction = float(tune_fraction)
        o.wait_timeout_s = float(wait_timeout_s)
        if stream is not None:
            o.stream = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        hs = (C.c_void_p * len(self.instances))(*[g.h for g in self.instances])
        b = C.c_void_p()
        rc = self._lib.parrep_batch_create(hs, len(self.instances), C.byref(o), C.byref(b))
        if rc != L.PARREP_OK:
            msg = self._lib.parrep_batch_last_error(None)
            raise ParRepError(rc, msg.decode() if msg else "")
        self.b = b

    def _check(self, rc):
        if rc != L.PARREP_OK:
            msg = self._lib.parrep_batch_last_error(self.b)
            raise ParRepError(rc, msg.decode() if msg else "")

    def run(self, T_end, seeds):
        n = len(self.instances)
        T = (C.c_double * n)(*[float(t) for t in (T_end if np.ndim(T_end) else [T_end] * n)])
        S = (C.c_uint64 * n)(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
        self._check(self._lib.parrep_batch_run(self.b, T, S))
        return self.info()

    def run_status(self, T_end, seeds) -> int:
        n = len(self.instances)
        T = (C.c_double * n)(*[float(t) for t in (T_end if np.ndim(T_end) else [T_end] * n)])
        S = (C.c_uint64 * n)(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
        return self._lib.parrep_batch_run(self.b, T, S)

    def status(self):
        out = (C.c_int32 * len(self.instances))()
        self._check(self._lib.parrep_batch_status(self.b, out))
        return list(out)

    def info(self) -> dict:
        i = L.parrep_batch_info()
        self._check(self._lib.parrep_batch_info_get(self.b, C.byref(i)))
        d = {k: getattr(i, k) for k, _ in i._fields_ if k != "pad"}
        d["f32_layout"] = {v: k for k, v in L.LAYOUTS.items() if k != "auto"}.get(d["f32_layout"])
        return d

    def close(self):
        if getattr(self, "b", None):
            self._lib.parrep_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats_dict(s) -> dict:
    d = {k: getattr(s, k) for k, _ in L.parrep_stats._fields_ if k != "pad"}
    d["x0"] = (s.x0[0], s.x0[1])
    d["x_final"] = (s.x_final[0], s.x_final[1])
    d["phase_cycles"] = {n: float(s.phase_cycles[i]) for i, n in enumerate(L.PHASES)}
    return d


class ParRepServer:
    """parrep_server_*: a request loop with continuous batching.  submit()
    returns an id at once; result() waits and returns the request's outputs."""

    def __init__(self, *, precision: str = "f32", block_threads: int = 0, replicas_per_block: int = 0,
                 ring: int = 4096, arena_bytes: int = 4 << 30, log_cap: int = 4096, idle_exit_s: float = 0.05,
                 wait_timeout_s: float = 10.0, f32_layout: str = "mixed"):
        self._lib = L.load()
        o = L.parrep_server_options()
        self._lib.parrep_server_default_options(C.byref(o))
        o.precision = L.PARREP_FP32 if precision == "f32" else L.PARREP_FP64
        o.block_threads = int(block_threads)
        o.replicas_per_block = int(replicas_per_block)
        o.ring = int(ring)
        o.f32_layout = L.LAYOUTS[f32_layout]
        o.arena_bytes = int(arena_bytes)
        o.log_cap = int(log_cap)
        o.idle_exit_s = float(idle_exit_s)
        o.wait_timeout_s = float(wait_timeout_s)
        s = C.c_void_p()
        rc = self._lib.parrep_server_create(C.byref(o), C.byref(s))
        if rc != L.PARREP_OK:
            msg = self._lib.parrep_server_last_error(None)
            raise ParRepError(rc, msg.decode() if msg else "")
        self.s = s
        self._meta = {}

    def _check(self, rc):
        if rc != L.PARREP_OK:
            msg = self._lib.parrep_server_last_error(self.s)
            raise ParRepError(rc, msg.decode() if msg else "")

    def submit(self, spec: dict, n_replicas: int, t_corr: float, t_phase: float, T_end: float, seed: int, *,
               x0=None, x0_uniform_hi: int = 0, thresh: str = "time", fv_group: int = 32, T_burn: float = 0.0,
               chunk_steps: int = 0, rer=None) -> int:
        r = L.parrep_request()
        r.net = make_network(spec, x0, x0_uniform_hi)
        r.regions = make_regions(spec)
        r.n_replicas = int(n_replicas)
        r.t_corr, r.t_phase = float(t_corr), float(t_phase)
        r.T_end, r.T_burn = float(T_end), float(T_burn)
        r.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        r.thresh_mode = L.PARREP_THRESH_STEPS if thresh == "steps" else L.PARREP_THRESH_TIME
        r.fv_group = int(fv_group)
        r.chunk_steps = int(chunk_steps)
        cp = None
        if rer is not None:
            cp = np.ascontiguousarray(rer, dtype=np.float64)
            r.n_cprime = cp.shape[0]
            r.c_prime = cp.ctypes.data
        rid = C.c_int64(0)
        self._check(self._lib.parrep_server_submit(self.s, C.byref(r), C.byref(rid)))
        nl = {"schlogl": 4, "toggle": 6, "genetic": 8}[spec["kind"]]
        hm = [spec["hist_max"]] if np.isscalar(spec["hist_max"]) else spec["hist_max"]
        self._meta[rid.value] = (int(np.prod([h + 1 for h in hm])), nl, 0 if cp is None else cp.shape[0])
        return rid.value

    def poll(self, rid: int) -> int:
        st = C.c_int32(0)
        self._check(self._lib.parrep_server_poll(self.s, int(rid), C.byref(st)))
        return st.value

    def wait(self, rid: int, timeout_s: float = 600.0):
        self._check(self._lib.parrep_server_wait(self.s, int(rid), float(timeout_s)))

    def result(self, rid: int, timeout_s: float = 600.0) -> dict:
        """Waits for the request, copies its outputs and releases it."""
        self.wait(rid, timeout_s)
        nb, nl, ncp = self._meta.pop(int(rid))
        st = L.parrep_stats()
        hist = np.zeros(nb)
        fim = np.zeros(nl * nl)
        rer = np.zeros(max(ncp, 1))
        lat = C.c_double(0.0)
        rc = self._lib.parrep_server_result(self.s, int(rid), C.byref(st), _buf(hist), nb, _buf(fim), _buf(rer),
                                            C.byref(lat))
        return {"status": rc, "stats": _stats_dict(st), "hist": hist, "fim": fim.reshape(nl, nl),
                "rer": rer[:ncp], "latency_s": lat.value}

    def stats(self) -> dict:
        s = L.parrep_server_stats()
        self._check(self._lib.parrep_server_stats_get(self.s, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "s", None):
            self._lib.parrep_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def parrep_ssa(spec: dict, n_traj: int, x0, T_end: float, seed: int, *, precision: str = "f64", stream=None,
               hist_out=None):
    """Plain SSA on the GPU.  Returns (histogram in time units, events, kernel ms)."""
    lib = L.load()
    net = make_network(spec, x0)
    nb = int(np.prod([h + 1 for h in ([spec["hist_max"]] if np.isscalar(spec["hist_max"]) else spec["hist_max"])]))
    hist = np.zeros(nb) if hist_out is None else hist_out
    ev = C.c_int64(0)
    ms = C.c_float(0.0)
    st = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib.parrep_ssa(C.byref(net), L.PARREP_FP32 if precision == "f32" else L.PARREP_FP64, int(n_traj),
                          float(T_end), int(seed), _buf(hist), nb, C.byref(ev), C.byref(ms), st))
    return hist, int(ev.value), float(ms.value)


def parrep_ssa_trace(spec: dict, n_traj: int, x0, T_end: float, seed: int, max_steps: int, *,
                     precision: str = "f64"):
    """Plain SSA with a record of every jump (the same counters as parrep_ssa).
    Returns (reactions (n_traj, max_steps), states (n_traj, max_steps, 2),
    holding times (n_traj, max_steps), jumps made (n_traj,), final states
    (n_traj, 2)); entries past a trajectory's jump count are unused."""
    lib = L.load()
    net = make_network(spec, x0)
    J = np.full((n_traj, max_steps), -1, dtype=np.int32)
    xs = np.zeros((n_traj, max_steps, 2), dtype=np.int32)
    tau = np.zeros((n_traj, max_steps))
    nj = np.zeros(n_traj, dtype=np.int64)
    xf = np.zeros((n_traj, 2), dtype=np.int32)
    _check(lib.parrep_ssa_trace(C.byref(net), L.PARREP_FP32 if precision == "f32" else L.PARREP_FP64, int(n_traj),
                                float(T_end), int(seed), int(max_steps), _buf(J), _buf(xs), _buf(tau), _buf(nj),
                                _buf(xf)))
    return J, xs, tau, nj, xf


def parrep_philox(ctr, key):
    """Device Philox4x32-10 on n counters (n x 4) and keys (n x 2)."""
    lib = L.load()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(lib.parrep_philox(_buf(ctr), _buf(key), len(ctr), _buf(out)))
    return out


def parrep_ssa_noalloc(spec: dict, n_traj: int, x0, T_end: float, seed: int, hist_out, *, precision: str = "f64",
                       stream=None):
    """parrep_ssa without device allocation (fixed scratch in the library).
    hist_out: float64 numpy array or torch tensor of n_bins.  Returns events."""
    lib = L.load()
    net = make_network(spec, x0)
    ev = C.c_int64(0)
    st = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    n = hist_out.numel() if hasattr(hist_out, "numel") else hist_out.size
    _check(lib.parrep_ssa_noalloc(C.byref(net), L.PARREP_FP32 if precision == "f32" else L.PARREP_FP64,
                                  int(n_traj), float(T_end), int(seed), _buf(hist_out), int(n), C.byref(ev), st))
    return int(ev.value)


def parrep_uq(handles, f, directions=None) -> dict:
    """Stationary UQ over independent completed runs (Sec. IV.B): the IAF of
    f, its stationary mean, the mean FIM with 95% half widths, and the
    information bounds sqrt(tau) sqrt(v^T I v) for the unit vectors (and for
    the rows of `directions`).  f: one value per histogram bin."""
    lib = L.load()
    hs = [h.h for h in handles]
    n = len(hs)
    arr = (C.c_void_p * max(n, 1))(*hs)
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    l = handles[0].L if n else 4
    dirs = None if directions is None else np.ascontiguousarray(directions, dtype=np.float64).reshape(-1, l)
    nd = 0 if dirs is None else len(dirs)
    db = np.zeros(max(nd, 1))
    Y = np.zeros(max(n, 1))
    r = L.parrep_uq_result()
    _check(lib.parrep_uq(arr, n, _buf(f), len(f), None if dirs is None else _buf(dirs), nd,
                         _buf(db) if nd else None, _buf(Y), C.byref(r)), hs[0] if n else None)
    out = dict(n_samples=r.n_samples, window=r.window, iaf=r.iaf, mean_f=r.mean_f, Y=Y[:n].copy(),
               fim=np.array(r.fim[: l * l]).reshape(l, l), fim_half_width=np.array(r.fim_half_width[: l * l]).reshape(l, l),
               bounds=np.array(r.bound[:l]))
    if nd:
        out["direction_bounds"] = db[:nd].copy()
    return out
