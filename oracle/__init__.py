"""CPU oracle for ParRep dynamics -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it, and it imports nothing from the product.

Contents:
  * ``parrep_oracle.c`` -- plain single-threaded C: Philox4x32-10, the
    Gillespie direct method, and Algorithm 1 of Wang & Plechac (arXiv
    1705.06807) step by step, in binary64 (and a binary32 propensity mode in
    which the reaction choice is taken in the same precision as the kernel's
    FP32 form).
  * ``exact.py`` -- exact references: birth-death product formula, truncated
    CME, quasi-stationary distributions, mean first passage times, closed-form
    FIM / relative entropy rate.
  * ``uq.py`` -- the Sec. IV.B estimators of the IAF, the stationary mean and
    the path-space FIM over independent runs, and the information bounds.
  * ``__init__.py`` (this file) -- builds the C file with gcc and wraps it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "parrep_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libparrep_oracle.so")
_lock = threading.Lock()
_lib = None

SCHLOGL, TOGGLE, GENETIC = 1, 2, 3
TIME, STEPS = 0, 1
F64, F32 = 0, 1
OR_OK, OR_EINVAL, OR_ENOMEM, OR_ERANGE = 0, -1, -2, -5


class Network(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("n_species", C.c_int32),
        ("c", C.c_double * 8),
        ("s", C.c_double * 4),
        ("hist_max", C.c_int32 * 2),
        ("n_regions", C.c_int32),
        ("reg_a", (C.c_int32 * 2) * 4),
        ("reg_b", C.c_int64 * 4),
    ]


class Config(C.Structure):
    _fields_ = [
        ("thresh_mode", C.c_int32),
        ("precision", C.c_int32),
        ("n_replicas", C.c_int64),
        ("fv_group", C.c_int32),
        ("x0_uniform_hi", C.c_int32),
        ("t_corr", C.c_double),
        ("t_phase", C.c_double),
        ("T_end", C.c_double),
        ("T_burn", C.c_double),
        ("seed", C.c_uint64),
        ("x0", C.c_int32 * 2),
    ]


class Cycle(C.Structure):
    _fields_ = [
        ("cycle", C.c_int64),
        ("W", C.c_int32),
        ("ended", C.c_int32),
        ("decorr_steps", C.c_int64),
        ("dephase_steps", C.c_int64),
        ("n_star", C.c_int64),
        ("k", C.c_int64),
        ("x_tilde", C.c_int32 * 2),
        ("T_s", C.c_double),
    ]


class Result(C.Structure):
    _fields_ = [
        ("T_s", C.c_double),
        ("events_decorr", C.c_int64),
        ("events_dephase", C.c_int64),
        ("events_parallel_useful", C.c_int64),
        ("cycles", C.c_int64),
        ("escapes", C.c_int64),
        ("x_final", C.c_int32 * 2),
        ("x0", C.c_int32 * 2),
        ("status", C.c_int32),
        ("pad", C.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE arithmetic, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.or_u01_f64.argtypes = [C.c_uint32, C.c_uint32]
            L.or_u01_f64.restype = C.c_double
            L.or_u01_f32.argtypes = [C.c_uint32]
            L.or_u01_f32.restype = C.c_float
            L.or_parrep_run.argtypes = [P(Network), P(Config), P(C.c_double), P(C.c_double), P(C.c_double),
                                        P(C.c_double), C.c_int32, P(C.c_double), P(Cycle), C.c_int64,
                                        P(C.c_int64), P(Result)]
            L.or_parrep_run_counted.argtypes = L.or_parrep_run.argtypes + [P(C.c_int64), P(C.c_int64)]
            L.or_dephase.argtypes = [P(Network), P(Config), P(C.c_int32), C.c_int32, C.c_uint32,
                                     P(C.c_int32), P(C.c_int64)]
            L.or_dephase.restype = C.c_int64
            L.or_parallel_from.argtypes = [P(Network), P(Config), P(C.c_int32), C.c_int32, C.c_uint32,
                                           C.c_int64, P(C.c_int64), P(C.c_int64), P(C.c_int32),
                                           P(C.c_double), P(C.c_double)]
            L.or_dephase_steps.argtypes = [P(Network), P(Config), P(C.c_int32)]
            L.or_dephase_steps.restype = C.c_int64
            L.or_ssa_run.argtypes = [P(Network), C.c_int32, C.c_int64, P(C.c_int32), C.c_double, C.c_uint64,
                                     P(C.c_double), P(C.c_int64), P(C.c_int32)]
            L.or_ssa_trace.argtypes = [P(Network), C.c_int32, P(C.c_int32), C.c_uint64, C.c_uint32, C.c_int64,
                                       P(C.c_int32), P(C.c_int32), P(C.c_double)]
            L.or_initial_state.argtypes = [P(Network), P(Config), P(C.c_int32)]
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---------------------------------------------------------------------------
# network / config constructors (plain data; no arithmetic of the method)
# ---------------------------------------------------------------------------
def network(spec: dict) -> Network:
    """Builds the C struct from a network spec dict (see the package's
    ``configs`` module for the field meanings)."""
    n = Network()
    n.kind = {"schlogl": SCHLOGL, "toggle": TOGGLE, "genetic": GENETIC}[spec["kind"]]
    n.n_species = 1 if n.kind == SCHLOGL else 2
    for i, v in enumerate(spec["c"]):
        n.c[i] = float(v)
    for i, v in enumerate(spec.get("s", [1.0, 1.0, 1.0, 1.0])):
        n.s[i] = float(v)
    hm = spec["hist_max"]
    hm = [hm] if np.isscalar(hm) else list(hm)
    n.hist_max[0] = int(hm[0])
    n.hist_max[1] = int(hm[1]) if len(hm) > 1 else 0
    regs = spec["regions"]
    n.n_regions = len(regs)
    for i, (a, b) in enumerate(regs):
        a = list(a) + [0] * (2 - len(a))
        n.reg_a[i][0] = int(a[0])
        n.reg_a[i][1] = int(a[1])
        n.reg_b[i] = int(b)
    return n


def config(n_replicas, t_corr, t_phase, T_end, seed, x0, *, thresh="time", precision="f64", fv_group=32,
           T_burn=0.0, x0_uniform_hi=0) -> Config:
    c = Config()
    c.thresh_mode = STEPS if thresh == "steps" else TIME
    c.precision = F32 if precision == "f32" else F64
    c.n_replicas = int(n_replicas)
    c.fv_group = int(fv_group)
    c.x0_uniform_hi = int(x0_uniform_hi)
    c.t_corr = float(t_corr)
    c.t_phase = float(t_phase)
    c.T_end = float(T_end)
    c.T_burn = float(T_burn)
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    x0 = [x0] if np.isscalar(x0) else list(x0)
    c.x0[0] = int(x0[0])
    c.x0[1] = int(x0[1]) if len(x0) > 1 else 0
    return c


def n_bins(spec: dict) -> int:
    hm = spec["hist_max"]
    hm = [hm] if np.isscalar(hm) else list(hm)
    return int(np.prod([h + 1 for h in hm]))


def n_params(spec: dict) -> int:
    return {"schlogl": 4, "toggle": 6, "genetic": 8}[spec["kind"]]


# ---------------------------------------------------------------------------
# wrappers
# ---------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def u01_f64(wa, wb) -> float:
    return lib().or_u01_f64(int(wa), int(wb))


def u01_f32(w) -> float:
    return lib().or_u01_f32(int(w))


def parrep_run(spec, n_replicas, t_corr, t_phase, T_end, seed, x0=None, *, thresh="time", precision="f64",
               fv_group=32, T_burn=0.0, x0_uniform_hi=0, rer_cprime=None, log_cap=100000, counts=False):
    """Runs Algorithm 1 to T_end.  Returns a dict with the pre- and post-burn-in
    histograms (time sums), the FIM and RER sums over [T_burn, T_end], the
    cycle log and the run statistics; with counts=True also the number of
    holding times added to each bin before and after T_burn."""
    net = network(spec)
    if x0 is None:
        x0 = [0, 0]
    cfg = config(n_replicas, t_corr, t_phase, T_end, seed, x0, thresh=thresh, precision=precision,
                 fv_group=fv_group, T_burn=T_burn, x0_uniform_hi=x0_uniform_hi)
    nb = n_bins(spec)
    l = n_params(spec)
    hpre = np.zeros(nb)
    hpost = np.zeros(nb)
    fim = np.zeros(l * l)
    if rer_cprime is None:
        rer_cprime = np.zeros((0, l))
    rer_cprime = np.ascontiguousarray(rer_cprime, dtype=np.float64).reshape(-1, l)
    rer = np.zeros(max(len(rer_cprime), 1))
    log = (Cycle * max(log_cap, 1))()
    log_n = C.c_int64(0)
    res = Result()
    cpre = np.zeros(nb, dtype=np.int64)
    cpost = np.zeros(nb, dtype=np.int64)
    rc = lib().or_parrep_run_counted(C.byref(net), C.byref(cfg), _ptr(hpre, C.c_double), _ptr(hpost, C.c_double),
                                     _ptr(fim, C.c_double), _ptr(rer_cprime, C.c_double), len(rer_cprime),
                                     _ptr(rer, C.c_double), log, log_cap, C.byref(log_n), C.byref(res),
                                     _ptr(cpre, C.c_int64) if counts else None,
                                     _ptr(cpost, C.c_int64) if counts else None)
    cycles = [
        dict(cycle=log[i].cycle, W=log[i].W, ended=log[i].ended, decorr_steps=log[i].decorr_steps,
             dephase_steps=log[i].dephase_steps, n_star=log[i].n_star, k=log[i].k,
             x_tilde=(log[i].x_tilde[0], log[i].x_tilde[1]), T_s=log[i].T_s)
        for i in range(log_n.value)
    ]
    return dict(status=rc, T_s=res.T_s, hist_pre=hpre, hist_post=hpost, fim=fim.reshape(l, l),
                rer=rer[: len(rer_cprime)], cycles=cycles, events_decorr=res.events_decorr,
                events_dephase=res.events_dephase, events_parallel_useful=res.events_parallel_useful,
                n_cycles=res.cycles, escapes=res.escapes, x_final=(res.x_final[0], res.x_final[1]),
                x0=(res.x0[0], res.x0[1]), **(dict(count_pre=cpre, count_post=cpost) if counts else {}))


def initial_state(spec, seed, x0, x0_uniform_hi) -> tuple:
    net = network(spec)
    cfg = config(1, 0, 0, 0, seed, x0, x0_uniform_hi=x0_uniform_hi)
    out = np.zeros(2, dtype=np.int32)
    lib().or_initial_state(C.byref(net), C.byref(cfg), _ptr(out, C.c_int32))
    return int(out[0]), int(out[1])


def dephase(spec, n_replicas, x_tilde, W, cycle, t_phase, seed, *, thresh="time", precision="f64",
            fv_group=32):
    """One dephasing stage from X~ in region W.  Returns (states (R,2), steps, events)."""
    net = network(spec)
    cfg = config(n_replicas, 0.0, t_phase, 0.0, seed, [0, 0], thresh=thresh, precision=precision,
                 fv_group=fv_group)
    xt = np.array(list(x_tilde) + [0] * (2 - len(x_tilde)), dtype=np.int32)
    xs = np.zeros((n_replicas, 2), dtype=np.int32)
    ev = C.c_int64(0)
    steps = lib().or_dephase(C.byref(net), C.byref(cfg), _ptr(xt, C.c_int32), int(W), int(cycle),
                             _ptr(xs, C.c_int32), C.byref(ev))
    return xs, int(steps), int(ev.value)


def parallel_from(spec, states, W, cycle, seed, *, precision="f64", max_steps=0, hist=None):
    """One parallel step from the given replica states, with no T_end.
    Returns (rc, N*, K, exit state, summed holding time of the contributions);
    ``hist`` (optional float64 array) receives the time-weighted histogram."""
    net = network(spec)
    states = np.ascontiguousarray(states, dtype=np.int32).reshape(-1, 2).copy()
    cfg = config(len(states), 0.0, 0.0, 0.0, seed, [0, 0], precision=precision)
    ns = C.c_int64(0)
    k = C.c_int64(0)
    xe = np.zeros(2, dtype=np.int32)
    ts = C.c_double(0.0)
    hp = _ptr(hist, C.c_double) if hist is not None else None
    rc = lib().or_parallel_from(C.byref(net), C.byref(cfg), _ptr(states, C.c_int32), int(W), int(cycle),
                                int(max_steps), C.byref(ns), C.byref(k), _ptr(xe, C.c_int32), C.byref(ts), hp)
    return rc, int(ns.value), int(k.value), (int(xe[0]), int(xe[1])), float(ts.value)


def dephase_steps(spec, x_tilde, t_phase, *, thresh="time"):
    net = network(spec)
    cfg = config(1, 0.0, t_phase, 0.0, 0, [0, 0], thresh=thresh)
    xt = np.array(list(x_tilde) + [0] * (2 - len(x_tilde)), dtype=np.int32)
    return int(lib().or_dephase_steps(C.byref(net), C.byref(cfg), _ptr(xt, C.c_int32)))


def ssa_run(spec, n_traj, x0, T_end, seed, *, precision="f64"):
    """Plain SSA for n_traj trajectories.  Returns (hist, events, final states)."""
    net = network(spec)
    x0 = np.array(([x0] if np.isscalar(x0) else list(x0)) + [0], dtype=np.int32)[:2].copy()
    hist = np.zeros(n_bins(spec))
    ev = C.c_int64(0)
    xf = np.zeros((n_traj, 2), dtype=np.int32)
    rc = lib().or_ssa_run(C.byref(net), F32 if precision == "f32" else F64, int(n_traj), _ptr(x0, C.c_int32),
                          float(T_end), int(seed), _ptr(hist, C.c_double), C.byref(ev), _ptr(xf, C.c_int32))
    if rc != 0:
        raise RuntimeError(f"oracle ssa_run failed: {rc}")
    return hist, int(ev.value), xf


def ssa_trace(spec, x0, seed, traj, n, *, precision="f64"):
    net = network(spec)
    x0 = np.array(([x0] if np.isscalar(x0) else list(x0)) + [0], dtype=np.int32)[:2].copy()
    J = np.zeros(n, dtype=np.int32)
    xs = np.zeros((n, 2), dtype=np.int32)
    tau = np.zeros(n)
    rc = lib().or_ssa_trace(C.byref(net), F32 if precision == "f32" else F64, _ptr(x0, C.c_int32), int(seed),
                            int(traj), int(n), _ptr(J, C.c_int32), _ptr(xs, C.c_int32), _ptr(tau, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle ssa_trace failed: {rc}")
    return J, xs, tau
