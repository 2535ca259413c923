"""ctypes binding of libfbg.so (include/fbg.h): argument marshalling only.

Every evaluation runs in the library's CUDA kernels; there is no CPU path.
If the in-tree library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1310_6978_b300.build`")

lib = ctypes.CDLL(LIB_PATH)

c_u64 = ctypes.c_uint64
c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t
c_char_p = ctypes.c_char_p

FBG_OK, FBG_EINVAL, FBG_EPARSE, FBG_ETOOBIG, FBG_ENOMEM, FBG_ECUDA, FBG_EJIT, FBG_ETIMEOUT, FBG_ECANCELLED, FBG_EBUSY = range(10)
STATUS_NAMES = ["FBG_OK", "FBG_EINVAL", "FBG_EPARSE", "FBG_ETOOBIG", "FBG_ENOMEM", "FBG_ECUDA", "FBG_EJIT",
                "FBG_ETIMEOUT", "FBG_ECANCELLED", "FBG_EBUSY"]

ENGINE_AUTO, ENGINE_JIT, ENGINE_INTERP = 0, 1, 2
OPT_ENGINE, OPT_PRUNE, OPT_REGS_LOG2, OPT_WARPS_LOG2, OPT_UNIT_BITS, OPT_LOOP_LEVEL_BITS, OPT_SEARCH_ORDER, \
    OPT_MIN_BLOCKS, OPT_STATS, OPT_INNER_BITS, OPT_SPLIT_ITEMS, OPT_POPC_COST, OPT_ORDER_SEED = range(1, 14)
MODE_COUNT, MODE_ENUMERATE = 0, 1
BATCH_GRAPH, BATCH_SPECIALIZE = 1, 2


class FbgStats(ctypes.Structure):
    _fields_ = [("n", c_int), ("domain_k", c_int), ("dag_nodes", c_i64), ("gates", c_i64), ("luts", c_i64),
                ("nlevels", c_int), ("lop3_per_level", c_i64 * 16), ("regs_log2", c_int), ("lane_bits", c_int),
                ("warp_bits", c_int), ("unit_bits", c_int), ("loop_bits", c_int * 8), ("interp_slots", c_int)]


class FbgExecStats(ctypes.Structure):
    _fields_ = [("level_iters", c_u64 * 16), ("lop3_executed", ctypes.c_double),
                ("lop3_nominal", ctypes.c_double), ("engine", c_int), ("lop3_uniform", ctypes.c_double)]


class FbgTuneResult(ctypes.Structure):
    _fields_ = [("best_ms", ctypes.c_double), ("trials", c_int), ("regs_log2", c_int), ("warps_log2", c_int),
                ("min_blocks", c_int), ("loop_level_bits", c_int), ("unit_bits", c_int), ("inner_bits", c_int),
                ("popc_cost", c_int), ("order_seed", c_int)]


class FbgServerOptions(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", c_u64), ("tick_units", c_u64), ("max_inflight", c_int),
                ("tick_assignments", c_u64), ("jit_min_n", c_int), ("jit_after", c_int), ("jit_max_programs", c_int)]


class FbgResult(ctypes.Structure):
    _fields_ = [("status", c_int), ("count", c_u64), ("written", c_u64), ("models", ctypes.POINTER(c_u64)),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


def _sig(name, res, *args):
    f = getattr(lib, name, None)
    if f is None:
        return None
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("fbg_compile", c_int, c_char_p, c_int, ctypes.POINTER(c_vp))
_sig("fbg_num_vars", c_int, c_vp)
_sig("fbg_var_name", c_int, c_vp, c_int, c_char_p, c_sz)
_sig("fbg_set_option", c_int, c_vp, c_int, c_i64)
_sig("fbg_program_stats", c_int, c_vp, ctypes.POINTER(FbgStats))
_sig("fbg_count", c_int, c_vp, c_vp, ctypes.POINTER(c_u64))
_sig("fbg_count_async", c_int, c_vp, c_vp, c_vp)
_sig("fbg_count_each", c_int, ctypes.POINTER(c_vp), c_sz, c_vp, c_vp)
_sig("fbg_count_noalloc", c_int, c_vp, c_vp, c_vp)
_sig("fbg_count_range", c_int, c_vp, c_vp, c_u64, c_u64, ctypes.POINTER(c_u64))
_sig("fbg_count_units", c_int, c_vp, c_vp, c_vp, c_u64)
_sig("fbg_debug_unit_trace", c_int, c_vp, c_vp, c_vp, c_u64)
_sig("fbg_schedule_units", c_int, c_vp, c_vp)
_sig("fbg_probe_lop3_rate", c_int, c_vp, ctypes.POINTER(ctypes.c_double))
_sig("fbg_debug_item_trace", c_int, c_vp, c_vp, c_vp, c_u64)
_sig("fbg_unit_vars", c_int, c_vp, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_u64))
_sig("fbg_truth_table", c_int, c_vp, c_vp, c_vp, c_sz)
_sig("fbg_enumerate_models", c_int, c_vp, c_vp, c_vp, c_sz, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64))
_sig("fbg_table_units", c_int, c_vp, c_int, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64))
_sig("fbg_truth_table_range", c_int, c_vp, c_vp, c_u64, c_u64, c_vp, c_sz)
_sig("fbg_enumerate_models_range", c_int, c_vp, c_vp, c_u64, c_u64, c_vp, c_sz, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64))
_sig("fbg_autotune", c_int, c_vp, c_vp, c_int, c_int, ctypes.POINTER(FbgTuneResult))
_sig("fbg_last_exec_stats", c_int, c_vp, ctypes.POINTER(FbgExecStats))
_sig("fbg_debug_host_times", c_int, c_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))
_sig("fbg_debug_host_caches", c_int, c_int, ctypes.POINTER(ctypes.c_uint64))
_sig("fbg_program_source", c_int, c_vp, c_int, c_char_p, ctypes.POINTER(c_sz))
_sig("fbg_debug_dump", c_int, c_vp, c_int, c_char_p, ctypes.POINTER(c_sz))
_sig("fbg_program_jit_log", c_char_p, c_vp)
_sig("fbg_program_free", None, c_vp)
_sig("fbg_last_error", c_char_p)
_sig("fbg_batch_create", c_int, ctypes.POINTER(c_vp), c_int, c_u64, c_int, ctypes.POINTER(c_vp))
_sig("fbg_batch_run", c_int, c_vp, c_vp)
_sig("fbg_batch_results", c_int, c_vp, c_vp, c_vp)
_sig("fbg_batch_info", c_int, c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64), ctypes.POINTER(c_int),
     ctypes.POINTER(c_int))
_sig("fbg_batch_program_kinds", c_int, c_vp, ctypes.POINTER(c_int))
_sig("fbg_debug_batch_source", c_int, ctypes.POINTER(c_vp), c_int, c_char_p, ctypes.POINTER(c_sz))
_sig("fbg_debug_nvrtc_compile", c_int, c_char_p, c_char_p, c_sz)
_sig("fbg_debug_batch_build", c_int, ctypes.POINTER(c_vp), c_int, ctypes.POINTER(c_int), c_char_p, c_sz)
_sig("fbg_batch_free", None, c_vp)
_sig("fbg_server_create", c_int, ctypes.POINTER(FbgServerOptions), ctypes.POINTER(c_vp))
_sig("fbg_server_submit", c_int, c_vp, c_char_p, c_int, c_int, c_u64, ctypes.POINTER(c_u64))
_sig("fbg_server_poll", c_int, c_vp, c_u64, ctypes.POINTER(FbgResult))
_sig("fbg_server_completed", c_int, c_vp, ctypes.POINTER(c_u64), c_sz, ctypes.POINTER(c_sz))
_sig("fbg_server_drain", c_int, c_vp, ctypes.c_double)
_sig("fbg_server_release", c_int, c_vp, c_u64)
_sig("fbg_server_stats", c_int, c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64), ctypes.POINTER(ctypes.c_double))
_sig("fbg_server_profile", c_int, c_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
     ctypes.POINTER(ctypes.c_double))
_sig("fbg_server_gpu_time", c_int, c_vp, ctypes.POINTER(ctypes.c_double))
_sig("fbg_server_jit_stats", c_int, c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64), ctypes.POINTER(ctypes.c_double))
_sig("fbg_server_free", None, c_vp)


class FbgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def check(status: int) -> None:
    if status != FBG_OK:
        raise FbgError(status, lib.fbg_last_error().decode(errors="replace"))
