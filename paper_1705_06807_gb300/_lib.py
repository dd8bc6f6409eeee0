"""ctypes binding of the C ABI in include/parrep.h (argument marshalling only).

The shared library is built in-tree by ``paper_1705_06807_gb300.build``.  If
it is missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libparrep.so")

PARREP_OK = 0
PARREP_EINVAL = -1
PARREP_ENOMEM = -2
PARREP_ECUDA = -3
PARREP_ETIMEOUT = -4
PARREP_F32_AUTO, PARREP_F32_STAGED, PARREP_F32_DIRECT, PARREP_F32_MIXED = 0, 1, 2, 3
LAYOUTS = {"auto": 0, "staged": 1, "direct": 2, "mixed": 3}
PARREP_ERANGE = -5
PARREP_ESTATE = -6
PARREP_SCHLOGL, PARREP_TOGGLE, PARREP_GENETIC = 1, 2, 3
PARREP_THRESH_TIME, PARREP_THRESH_STEPS = 0, 1
PARREP_FP64, PARREP_FP32 = 0, 1

ERRORS = {PARREP_EINVAL: "EINVAL", PARREP_ENOMEM: "ENOMEM", PARREP_ECUDA: "ECUDA", PARREP_ETIMEOUT: "ETIMEOUT",
          PARREP_ERANGE: "ERANGE", PARREP_ESTATE: "ESTATE"}


class parrep_network(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_species", C.c_int32), ("c", C.c_double * 8), ("s", C.c_double * 4),
                ("x0", C.c_int32 * 2), ("x0_uniform_hi", C.c_int32), ("hist_max", C.c_int32 * 2)]


class parrep_regions(C.Structure):
    _fields_ = [("n", C.c_int32), ("a", (C.c_int32 * 2) * 4), ("b", C.c_int64 * 4)]


class parrep_options(C.Structure):
    _fields_ = [("thresh_mode", C.c_int32), ("precision", C.c_int32), ("fv_group", C.c_int32),
                ("block_threads", C.c_int32), ("chunk_steps", C.c_int32), ("debug_stall_barrier", C.c_int32),
                ("serial_stages", C.c_int32), ("max_blocks", C.c_int32), ("f32_layout", C.c_int32),
                ("T_burn", C.c_double), ("wait_timeout_s", C.c_double), ("stream", C.c_void_p)]


class parrep_stats(C.Structure):
    _fields_ = [("T_s", C.c_double), ("events_decorr", C.c_int64), ("events_dephase", C.c_int64),
                ("events_parallel_useful", C.c_int64), ("events_parallel_executed", C.c_int64),
                ("events_replay", C.c_int64), ("cycles", C.c_int64), ("escapes", C.c_int64),
                ("chunks", C.c_int64), ("special_chunks", C.c_int64), ("x0", C.c_int32 * 2),
                ("x_final", C.c_int32 * 2), ("status", C.c_int32), ("grid_blocks", C.c_int32),
                ("block_threads", C.c_int32), ("chunk_steps", C.c_int32), ("kernel_ms", C.c_float),
                ("pad", C.c_float), ("phase_cycles", C.c_double * 12)]

class parrep_batch_options(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("replicas_per_block", C.c_int32), ("autotune", C.c_int32),
                ("use_graph", C.c_int32), ("f32_layout", C.c_int32), ("tune_fraction", C.c_double),
                ("wait_timeout_s", C.c_double), ("stream", C.c_void_p)]


class parrep_batch_info(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("replicas_per_block", C.c_int32), ("grid_blocks", C.c_int32),
                ("n_items", C.c_int32), ("graph", C.c_int32), ("tuned_trials", C.c_int32),
                ("f32_layout", C.c_int32), ("pad", C.c_int32), ("kernel_ms", C.c_float), ("tune_ms", C.c_float), ("est_makespan", C.c_double),
                ("est_balance", C.c_double)]


class parrep_server_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("block_threads", C.c_int32), ("replicas_per_block", C.c_int32),
                ("ring", C.c_int32), ("f32_layout", C.c_int32), ("arena_bytes", C.c_int64), ("log_cap", C.c_int64),
                ("idle_exit_s", C.c_double), ("wait_timeout_s", C.c_double)]


class parrep_request(C.Structure):
    _fields_ = [("net", parrep_network), ("regions", parrep_regions), ("n_replicas", C.c_int64),
                ("t_corr", C.c_double), ("t_phase", C.c_double), ("T_end", C.c_double), ("T_burn", C.c_double),
                ("seed", C.c_uint64), ("thresh_mode", C.c_int32), ("fv_group", C.c_int32),
                ("chunk_steps", C.c_int32), ("n_cprime", C.c_int32), ("c_prime", C.c_void_p)]


class parrep_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("released", C.c_int64), ("launches", C.c_int64), ("queued", C.c_int64), ("running", C.c_int64),
                ("arena_bytes", C.c_int64), ("arena_used", C.c_int64), ("grid_blocks", C.c_int32),
                ("block_threads", C.c_int32)]


PARREP_REQ_QUEUED, PARREP_REQ_RUNNING, PARREP_REQ_DONE = 0, 1, 2

PHASES = ["decorrelation", "dephasing", "draw", "chain", "account", "barrier", "special", "vote", "dec_draw",
          "dec_chain", "dec_times", "dec_commit"]


class parrep_cycle(C.Structure):
    _fields_ = [("cycle", C.c_int64), ("W", C.c_int32), ("ended", C.c_int32), ("decorr_steps", C.c_int64),
                ("dephase_steps", C.c_int64), ("n_star", C.c_int64), ("k", C.c_int64), ("x_tilde", C.c_int32 * 2),
                ("T_s", C.c_double)]


class parrep_uq_result(C.Structure):
    _fields_ = [("n_samples", C.c_int32), ("n_params", C.c_int32), ("window", C.c_double), ("iaf", C.c_double),
                ("mean_f", C.c_double), ("fim", C.c_double * 64), ("fim_half_width", C.c_double * 64),
                ("bound", C.c_double * 8)]


EXPORTS = ["parrep_default_options", "parrep_create", "parrep_set_options", "parrep_run", "parrep_n_bins",
           "parrep_histogram", "parrep_histogram_raw", "parrep_fim", "parrep_rer", "parrep_stats_get",
           "parrep_cycle_log", "parrep_dephase", "parrep_destroy", "parrep_last_error", "parrep_ssa",
           "parrep_philox", "parrep_ssa_noalloc", "parrep_ssa_trace", "parrep_batch_default_options", "parrep_batch_create",
           "parrep_batch_run", "parrep_batch_status", "parrep_batch_info_get", "parrep_batch_destroy",
           "parrep_batch_last_error", "parrep_server_default_options", "parrep_server_create",
           "parrep_server_submit", "parrep_server_poll", "parrep_server_wait", "parrep_server_result",
           "parrep_server_stats_get", "parrep_server_destroy", "parrep_server_last_error", "parrep_uq"]

_lib = None


def load():
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run paper_1705_06807_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    L.parrep_default_options.argtypes = [P(parrep_options)]
    L.parrep_default_options.restype = None
    L.parrep_create.argtypes = [P(parrep_network), C.c_int64, P(parrep_regions), C.c_double, C.c_double, P(vp)]
    L.parrep_set_options.argtypes = [vp, P(parrep_options)]
    L.parrep_run.argtypes = [vp, C.c_double, C.c_uint64]
    L.parrep_n_bins.argtypes = [vp]
    L.parrep_n_bins.restype = C.c_int64
    L.parrep_histogram.argtypes = [vp, vp, C.c_int64]
    L.parrep_histogram_raw.argtypes = [vp, vp, vp, C.c_int64]
    L.parrep_fim.argtypes = [vp, vp, C.c_int32]
    L.parrep_rer.argtypes = [vp, vp, C.c_int32, vp]
    L.parrep_stats_get.argtypes = [vp, P(parrep_stats)]
    L.parrep_cycle_log.argtypes = [vp, P(parrep_cycle), C.c_int64, P(C.c_int64)]
    L.parrep_dephase.argtypes = [vp, P(C.c_int32), C.c_int32, C.c_uint32, C.c_uint64, vp]
    L.parrep_destroy.argtypes = [vp]
    L.parrep_destroy.restype = None
    L.parrep_last_error.argtypes = [vp]
    L.parrep_last_error.restype = C.c_char_p
    L.parrep_ssa.argtypes = [P(parrep_network), C.c_int32, C.c_int64, C.c_double, C.c_uint64, vp, C.c_int64,
                             P(C.c_int64), P(C.c_float), vp]
    L.parrep_philox.argtypes = [vp, vp, C.c_int64, vp]
    L.parrep_ssa_trace.argtypes = [P(parrep_network), C.c_int32, C.c_int64, C.c_double, C.c_uint64, C.c_int64, vp,
                                   vp, vp, vp, vp]
    L.parrep_ssa_noalloc.argtypes = [P(parrep_network), C.c_int32, C.c_int64, C.c_double, C.c_uint64, vp,
                                     C.c_int64, P(C.c_int64), vp]
    L.parrep_batch_default_options.argtypes = [P(parrep_batch_options)]
    L.parrep_batch_default_options.restype = None
    L.parrep_batch_create.argtypes = [P(vp), C.c_int32, P(parrep_batch_options), P(vp)]
    L.parrep_batch_run.argtypes = [vp, P(C.c_double), P(C.c_uint64)]
    L.parrep_batch_status.argtypes = [vp, P(C.c_int32)]
    L.parrep_batch_info_get.argtypes = [vp, P(parrep_batch_info)]
    L.parrep_batch_destroy.argtypes = [vp]
    L.parrep_batch_destroy.restype = None
    L.parrep_batch_last_error.argtypes = [vp]
    L.parrep_batch_last_error.restype = C.c_char_p
    L.parrep_server_default_options.argtypes = [P(parrep_server_options)]
    L.parrep_server_default_options.restype = None
    L.parrep_server_create.argtypes = [P(parrep_server_options), P(vp)]
    L.parrep_server_submit.argtypes = [vp, P(parrep_request), P(C.c_int64)]
    L.parrep_server_poll.argtypes = [vp, C.c_int64, P(C.c_int32)]
    L.parrep_server_wait.argtypes = [vp, C.c_int64, C.c_double]
    L.parrep_server_result.argtypes = [vp, C.c_int64, P(parrep_stats), vp, C.c_int64, vp, vp, P(C.c_double)]
    L.parrep_server_stats_get.argtypes = [vp, P(parrep_server_stats)]
    L.parrep_server_destroy.argtypes = [vp]
    L.parrep_server_destroy.restype = None
    L.parrep_server_last_error.argtypes = [vp]
    L.parrep_server_last_error.restype = C.c_char_p
    L.parrep_uq.argtypes = [P(vp), C.c_int32, vp, C.c_int64, vp, C.c_int32, vp, vp, P(parrep_uq_result)]
    for name in EXPORTS:
        if name not in ("parrep_default_options", "parrep_n_bins", "parrep_destroy", "parrep_last_error",
                        "parrep_batch_default_options", "parrep_batch_destroy", "parrep_batch_last_error",
                        "parrep_server_default_options", "parrep_server_destroy", "parrep_server_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L
