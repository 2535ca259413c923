"""Free-Boolean-generator model counting on B300 (sm_103a).

Python binding of libfbg.so (include/fbg.h).  A theory is compiled on the host
(``compile``); counts, truth tables and model lists are computed by the
library's CUDA kernels.  PyTorch is used only to hold device buffers and
streams: pass ``torch.cuda.Stream`` objects (or None for the current stream)
and CUDA tensors (their ``data_ptr()`` is handed to the library).
"""
from __future__ import annotations

import ctypes
import json

__all__ = ["compile", "Program", "Batch", "Server", "FbgError", "read_counts"]

MASK64 = (1 << 64) - 1


def read_counts(dev_words) -> "list[int]":
    """The unsigned 64-bit counts that ``count_async`` (or ``count_units``)
    wrote into a torch.int64 tensor, as Python ints: the tensor's elements are
    read as bit patterns, so a count of 2^63 (n = 63) is not negative."""
    return [int(v) & MASK64 for v in dev_words.detach().reshape(-1).cpu().tolist()]


def _L():
    from . import _lib
    return _lib


def __getattr__(name):
    if name == "FbgError":
        return _L().FbgError
    raise AttributeError(name)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(t) -> int:
    return t if isinstance(t, int) else int(t.data_ptr())


class Program:
    """A compiled theory (fbg_compile).  n = number of propositional letters."""

    def __init__(self, text: str, domain_k: int = 1):
        L = _L()
        h = ctypes.c_void_p()
        L.check(L.lib.fbg_compile(text.encode(), int(domain_k), ctypes.byref(h)))
        self._h = h
        self._L = L
        self.text = text
        self.k = domain_k
        self.n = L.lib.fbg_num_vars(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.lib.fbg_program_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_option(self, option: int, value: int) -> "Program":
        self._L.check(self._L.lib.fbg_set_option(self._h, option, int(value)))
        return self

    def var_name(self, i: int) -> str:
        buf = ctypes.create_string_buffer(128)
        self._L.check(self._L.lib.fbg_var_name(self._h, i, buf, 128))
        return buf.value.decode()

    def stats(self):
        s = self._L.FbgStats()
        self._L.check(self._L.lib.fbg_program_stats(self._h, ctypes.byref(s)))
        return s

    def count(self, stream=None) -> int:
        out = ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_count(self._h, _stream_ptr(stream), ctypes.byref(out)))
        return out.value

    def count_async(self, dev_out, stream=None) -> None:
        """fbg_count_async: the count into ``dev_out`` (one 64-bit device
        element, e.g. a torch.int64 tensor) without waiting; read it back
        with ``read_counts`` (an unsigned 64-bit value)."""
        self._L.check(self._L.lib.fbg_count_async(self._h, _stream_ptr(stream), _ptr(dev_out)))

    def count_noalloc(self, dev_out, stream=None) -> None:
        """fbg_count_noalloc: the count into device memory ``dev_out`` (one
        64-bit element) with no device allocation by the library."""
        self._L.check(self._L.lib.fbg_count_noalloc(self._h, _stream_ptr(stream), _ptr(dev_out)))

    def unit_vars(self):
        vars_ = (ctypes.c_int * 64)()
        nv = ctypes.c_int()
        nu = ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_unit_vars(self._h, vars_, 64, ctypes.byref(nv), ctypes.byref(nu)))
        return [vars_[i] for i in range(nv.value)], nu.value

    def count_range(self, unit_begin: int, unit_end: int, stream=None) -> int:
        """fbg_count_range: models among units [unit_begin, unit_end)."""
        out = ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_count_range(self._h, _stream_ptr(stream), unit_begin, unit_end, ctypes.byref(out)))
        return out.value

    def count_units(self, dev_counts, stream=None) -> None:
        self._L.check(self._L.lib.fbg_count_units(self._h, _stream_ptr(stream), _ptr(dev_counts), dev_counts.numel()))

    def schedule_units(self, stream=None) -> "Program":
        """fbg_schedule_units: time every (unit, warp slice) item once and hand
        items out longest first in later full-range counts."""
        self._L.check(self._L.lib.fbg_schedule_units(self._h, _stream_ptr(stream)))
        return self

    def debug_host_times(self):
        """fbg_debug_host_times: (seconds building kernels, seconds in
        fbg_count outside builds) spent by this program so far."""
        b, c = ctypes.c_double(), ctypes.c_double()
        self._L.check(self._L.lib.fbg_debug_host_times(self._h, ctypes.byref(b), ctypes.byref(c)))
        return b.value, c.value

    def debug_item_trace(self, dev_ns, stream=None) -> None:
        """fbg_debug_item_trace: nanoseconds per (unit, warp slice) item."""
        self._L.check(self._L.lib.fbg_debug_item_trace(self._h, _stream_ptr(stream), _ptr(dev_ns), dev_ns.numel()))

    def debug_unit_trace(self, dev_trace, stream=None) -> None:
        """fbg_debug_unit_trace: per unit u, dev_trace[2u] = warp-nanoseconds
        spent and dev_trace[2u+1] = earliest start (GPU timer, ns); dev_trace
        holds 2 * nunits int64 words."""
        self._L.check(self._L.lib.fbg_debug_unit_trace(self._h, _stream_ptr(stream), _ptr(dev_trace),
                                                       dev_trace.numel() // 2))

    def table_words(self) -> int:
        return 1 if self.n <= 6 else 1 << (self.n - 6)

    def truth_table(self, dev_words, stream=None) -> None:
        self._L.check(self._L.lib.fbg_truth_table(self._h, _stream_ptr(stream), _ptr(dev_words), dev_words.numel()))

    def enumerate_models(self, dev_models, cap: int | None = None, stream=None):
        cap = dev_models.numel() if cap is None else cap
        total = ctypes.c_uint64()
        written = ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_enumerate_models(self._h, _stream_ptr(stream), _ptr(dev_models), cap,
                                                       ctypes.byref(total), ctypes.byref(written)))
        return total.value, written.value

    def table_units(self, mode: int = 1):
        """fbg_table_units: (units, 64-bit words per unit) of the table
        (mode 1) or model-list (mode 2) layout of the specialised kernel."""
        nu, wpu = ctypes.c_uint64(), ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_table_units(self._h, mode, ctypes.byref(nu), ctypes.byref(wpu)))
        return nu.value, wpu.value

    def truth_table_range(self, unit_begin: int, unit_end: int, dev_words, stream=None) -> None:
        """fbg_truth_table_range: the table words of units [unit_begin, unit_end)."""
        self._L.check(self._L.lib.fbg_truth_table_range(self._h, _stream_ptr(stream), unit_begin, unit_end,
                                                        _ptr(dev_words), dev_words.numel()))

    def enumerate_models_range(self, unit_begin: int, unit_end: int, dev_models, cap: int | None = None,
                               stream=None):
        """fbg_enumerate_models_range: (total, written) for the models among
        units [unit_begin, unit_end), ascending, the first `cap` stored."""
        cap = dev_models.numel() if cap is None else cap
        total, written = ctypes.c_uint64(), ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_enumerate_models_range(self._h, _stream_ptr(stream), unit_begin, unit_end,
                                                             _ptr(dev_models), cap, ctypes.byref(total),
                                                             ctypes.byref(written)))
        return total.value, written.value

    def autotune(self, mode: int = 0, reps: int = 3, stream=None) -> dict:
        """fbg_autotune: search the kernel shape; the program keeps the best."""
        r = self._L.FbgTuneResult()
        self._L.check(self._L.lib.fbg_autotune(self._h, _stream_ptr(stream), mode, reps, ctypes.byref(r)))
        return {"best_ms": r.best_ms, "trials": r.trials, "regs_log2": r.regs_log2, "warps_log2": r.warps_log2,
                "min_blocks": r.min_blocks, "loop_level_bits": r.loop_level_bits, "unit_bits": r.unit_bits,
                "inner_bits": r.inner_bits, "popc_cost": r.popc_cost, "order_seed": r.order_seed}

    def apply_shape(self, shape: dict) -> "Program":
        """Set the kernel-shape options recorded by ``autotune``."""
        L = self._L
        for key, opt in (("regs_log2", L.OPT_REGS_LOG2), ("warps_log2", L.OPT_WARPS_LOG2),
                         ("min_blocks", L.OPT_MIN_BLOCKS), ("loop_level_bits", L.OPT_LOOP_LEVEL_BITS),
                         ("inner_bits", L.OPT_INNER_BITS), ("popc_cost", L.OPT_POPC_COST),
                         ("order_seed", L.OPT_ORDER_SEED),
                         ("unit_bits", L.OPT_UNIT_BITS)):
            if key in shape:
                self.set_option(opt, shape[key])
        return self

    def exec_stats(self):
        s = self._L.FbgExecStats()
        self._L.check(self._L.lib.fbg_last_exec_stats(self._h, ctypes.byref(s)))
        return s

    def source(self, mode: int = 0) -> str:
        n = ctypes.c_size_t()
        self._L.check(self._L.lib.fbg_program_source(self._h, mode, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._L.check(self._L.lib.fbg_program_source(self._h, mode, buf, ctypes.byref(n)))
        return buf.value.decode()

    def debug_dump(self, which: int) -> dict:
        n = ctypes.c_size_t()
        self._L.check(self._L.lib.fbg_debug_dump(self._h, which, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._L.check(self._L.lib.fbg_debug_dump(self._h, which, buf, ctypes.byref(n)))
        return json.loads(buf.value.decode())

    def jit_log(self) -> str:
        return self._L.lib.fbg_program_jit_log(self._h).decode(errors="replace")


def compile(text: str, domain_k: int = 1) -> Program:   # noqa: A001 - mirrors fbg_compile
    return Program(text, domain_k)


class Batch:
    """Many programs counted in one persistent launch (fbg_batch_*)."""

    def __init__(self, programs, max_item_units: int = 0, use_graph: bool = True, specialize: bool = True):
        L = _L()
        self._L = L
        self.programs = list(programs)
        arr = (ctypes.c_void_p * len(self.programs))(*[p.handle.value for p in self.programs])
        h = ctypes.c_void_p()
        flags = (L.BATCH_GRAPH if use_graph else 0) | (L.BATCH_SPECIALIZE if specialize else 0)
        L.check(L.lib.fbg_batch_create(arr, len(self.programs), max_item_units, flags, ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.lib.fbg_batch_free(h)
            self._h = None

    def run(self, stream=None) -> None:
        self._L.check(self._L.lib.fbg_batch_run(self._h, _stream_ptr(stream)))

    def results(self, stream=None):
        import numpy as np
        out = np.zeros(len(self.programs), dtype=np.uint64)
        self._L.check(self._L.lib.fbg_batch_results(self._h, _stream_ptr(stream), out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def program_kinds(self):
        out = (ctypes.c_int * len(self.programs))()
        self._L.check(self._L.lib.fbg_batch_program_kinds(self._h, out))
        return [out[i] for i in range(len(self.programs))]

    def info(self):
        items, units, grid, spec = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int(), ctypes.c_int()
        self._L.check(self._L.lib.fbg_batch_info(self._h, ctypes.byref(items), ctypes.byref(units), ctypes.byref(grid),
                                                 ctypes.byref(spec)))
        return {"items": items.value, "units": units.value, "grid": grid.value, "specialized": spec.value}


def count_each(programs, dev_out, stream=None) -> None:
    """fbg_count_each: one count launch per program, back to back on the
    stream, into dev_out[i] (a device int64 tensor of len(programs))."""
    L = _L()
    arr = (ctypes.c_void_p * len(programs))(*[p.handle.value for p in programs])
    L.check(L.lib.fbg_count_each(arr, len(programs), _stream_ptr(stream), _ptr(dev_out)))


def host_caches(clear: bool = False) -> dict:
    """fbg_debug_host_caches: hits, misses and entries of the host compile
    caches (optionally emptied first)."""
    L = _L()
    out = (ctypes.c_uint64 * 9)()
    L.check(L.lib.fbg_debug_host_caches(1 if clear else 0, out))
    names = ("compile", "jit_build", "interp_build")
    return {nm: {"hits": out[3 * i], "misses": out[3 * i + 1], "entries": out[3 * i + 2]} for i, nm in enumerate(names)}


def probe_lop3_rate(stream=None) -> float:
    """fbg_probe_lop3_rate: measured lop3.b32 issue rate of this GPU (T/s)."""
    L = _L()
    t = ctypes.c_double()
    L.check(L.lib.fbg_probe_lop3_rate(_stream_ptr(stream), ctypes.byref(t)))
    return t.value


def batch_source(programs) -> str:
    """fbg_debug_batch_source: NVRTC sources of the batch's specialised kernels."""
    L = _L()
    arr = (ctypes.c_void_p * len(programs))(*[p.handle.value for p in programs])
    n = ctypes.c_size_t()
    L.check(L.lib.fbg_debug_batch_source(arr, len(programs), None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    L.check(L.lib.fbg_debug_batch_source(arr, len(programs), buf, ctypes.byref(n)))
    return buf.value.decode()


def batch_build_check(programs):
    """fbg_debug_batch_build: compile the batch's specialised kernels without a
    device; returns (ok, number that compile, log)."""
    L = _L()
    arr = (ctypes.c_void_p * len(programs))(*[p.handle.value for p in programs])
    spec = ctypes.c_int()
    log = ctypes.create_string_buffer(1 << 16)
    st = L.lib.fbg_debug_batch_build(arr, len(programs), ctypes.byref(spec), log, 1 << 16)
    return st == L.FBG_OK, spec.value, log.value.decode(errors="replace")


def nvrtc_check(body: str):
    """fbg_debug_nvrtc_compile: compile a kernel body with NVRTC (no device);
    returns (ok, log)."""
    L = _L()
    log = ctypes.create_string_buffer(1 << 16)
    st = L.lib.fbg_debug_nvrtc_compile(body.encode(), log, 1 << 16)
    return st == L.FBG_OK, log.value.decode(errors="replace")


class Server:
    """Continuous-batching request loop (fbg_server_*)."""

    def __init__(self, mem_budget_bytes: int = 0, tick_units: int = 0, max_inflight: int = 0,
                 tick_assignments: int = 0, jit_min_n: int = 0, jit_after: int = 0, jit_max_programs: int = 0):
        """Options as fbg_server_options (0 = the library's default).  jit_min_n
        < 0 keeps every request on the interpreter; otherwise count requests
        of a recurring text with at least jit_min_n letters (default 30) move
        to a specialised kernel compiled in the background after jit_after
        submissions (default 2)."""
        L = _L()
        self._L = L
        o = L.FbgServerOptions(mem_budget_bytes, tick_units, max_inflight, tick_assignments, jit_min_n, jit_after,
                               jit_max_programs)
        h = ctypes.c_void_p()
        L.check(L.lib.fbg_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.lib.fbg_server_free(h)
            self._h = None

    def submit(self, text: str, domain_k: int, mode: int = 0, cap: int = 0) -> int:
        rid = ctypes.c_uint64()
        self._L.check(self._L.lib.fbg_server_submit(self._h, text.encode(), int(domain_k), mode, cap, ctypes.byref(rid)))
        return rid.value

    def poll(self, rid: int, models: bool = True):
        """The result of a finished request (None while it runs); with
        models=False the model list is left out (its length is "written")."""
        r = self._L.FbgResult()
        st = self._L.lib.fbg_server_poll(self._h, rid, ctypes.byref(r))
        if st == self._L.FBG_EBUSY:
            return None
        self._L.check(st)
        if models and r.written:
            import numpy as np
            models = np.ctypeslib.as_array(r.models, shape=(r.written,)).tolist()
        else:
            models = []
        return {"status": r.status, "count": r.count, "written": r.written, "models": models,
                "submit_s": r.submit_s, "admit_s": r.admit_s, "done_s": r.done_s}

    def completed(self, max_ids: int = 4096):
        """fbg_server_completed: ids of requests finished since the last call."""
        buf = (ctypes.c_uint64 * max_ids)()
        n = ctypes.c_size_t()
        self._L.check(self._L.lib.fbg_server_completed(self._h, buf, max_ids, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    def drain(self, timeout_s: float = 0.0) -> None:
        self._L.check(self._L.lib.fbg_server_drain(self._h, timeout_s))

    def release(self, rid: int) -> None:
        self._L.check(self._L.lib.fbg_server_release(self._h, rid))

    def stats(self):
        t, l, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
        self._L.check(self._L.lib.fbg_server_stats(self._h, ctypes.byref(t), ctypes.byref(l), ctypes.byref(b)))
        a, c, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._L.check(self._L.lib.fbg_server_profile(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(e)))
        g = ctypes.c_double()
        self._L.check(self._L.lib.fbg_server_gpu_time(self._h, ctypes.byref(g)))
        jp, jr, jc = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
        self._L.check(self._L.lib.fbg_server_jit_stats(self._h, ctypes.byref(jp), ctypes.byref(jr), ctypes.byref(jc)))
        return {"ticks": t.value, "launches": l.value, "busy_s": b.value, "admit_s": a.value, "count_s": c.value,
                "enum_s": e.value, "gpu_s": g.value, "jit_programs": jp.value, "jit_requests": jr.value,
                "jit_compile_s": jc.value}
