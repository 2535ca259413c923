"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product.

The oracle computes the plain definition of the method (Prop. 2.2, Sec. 2.3):
bit j of the vector t(b_1..b_n) is the value of the theory under the
valuation mu_j, where variable x_i takes bit i of j (the generator matrix of
Sec. 2.2 with the index order flipped).  For each j it model-checks the
quantified formula on the structure h(mu_j) of Sec. 3.2 with plain booleans
(``oracle.c``); the model count l_{T,n} is the number of ones (Sec. 3.2).

``counters`` holds independent counters (backtracking / brute force over
structures, written without any formula text) that pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, OpenMP for the timed
    multi-core count only)."""
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "counters.c")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, *srcs])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, vp, c = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_char_p
            lib.oracle_parse.argtypes = [c, ctypes.c_int, ctypes.POINTER(vp), c, ctypes.c_int]
            lib.oracle_parse.restype = ctypes.c_int
            lib.oracle_free.argtypes = [vp]
            lib.oracle_num_vars.argtypes = [vp]
            lib.oracle_num_letters.argtypes = [vp]
            lib.oracle_eval.argtypes = [vp, u64]
            lib.oracle_eval.restype = ctypes.c_int
            lib.oracle_range.argtypes = [vp, u64, u64, ctypes.POINTER(u64), vp, vp, u64, ctypes.POINTER(u64)]
            lib.oracle_count_cube.argtypes = [vp, u64, u64]
            lib.oracle_count_cube.restype = u64
            lib.oracle_count_cube_par.argtypes = [vp, u64, u64, ctypes.c_int]
            lib.oracle_count_cube_par.restype = u64
            lib.oracle_cube_size.argtypes = [ctypes.c_int]
            lib.oracle_cube_size.restype = u64
            lib.oracle_count_par.argtypes = [vp, u64, u64, ctypes.c_int]
            lib.oracle_count_par.restype = u64
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.counter_transitive.argtypes = [ctypes.c_int]
            lib.counter_transitive.restype = u64
            lib.counter_posets.argtypes = [ctypes.c_int]
            lib.counter_posets.restype = u64
            lib.counter_posets_special.argtypes = [ctypes.c_int]
            lib.counter_posets_special.restype = u64
            lib.counter_triangle_free.argtypes = [ctypes.c_int]
            lib.counter_triangle_free.restype = u64
            _lib = lib
    return _lib


class OracleError(ValueError):
    pass


class Theory:
    """A parsed theory; every query walks the formula once per assignment."""

    def __init__(self, text: str, k: int = 1):
        lib = _load()
        h = ctypes.c_void_p()
        err = ctypes.create_string_buffer(512)
        if lib.oracle_parse(text.encode(), int(k), ctypes.byref(h), err, 512) != 0:
            raise OracleError(err.value.decode())
        self._h = h
        self._lib = lib
        self.n = lib.oracle_num_vars(h)
        self.k = k

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.oracle_free(h)
            self._h = None

    def eval(self, j: int) -> int:
        return self._lib.oracle_eval(self._h, j)

    def count(self, lo: int = 0, hi: int | None = None) -> int:
        hi = (1 << self.n) if hi is None else hi
        out = ctypes.c_uint64()
        self._lib.oracle_range(self._h, lo, hi, ctypes.byref(out), None, None, 0, None)
        return out.value

    def table(self) -> "list[int]":
        """Truth table as u64 words: bit j at word j>>6, bit j&63; for n<6 the
        bits >= 2^n of the single word stay 0."""
        import numpy as np
        nw = max(1, (1 << self.n) >> 6)
        words = np.zeros(nw, dtype=np.uint64)
        out = ctypes.c_uint64()
        self._lib.oracle_range(self._h, 0, 1 << self.n, ctypes.byref(out),
                               words.ctypes.data_as(ctypes.c_void_p), None, 0, None)
        return words

    def models(self, cap: int, lo: int = 0, hi: int | None = None):
        """First ``cap`` models in ascending j, and the exact total."""
        import numpy as np
        hi = (1 << self.n) if hi is None else hi
        buf = np.zeros(max(1, cap), dtype=np.uint64)
        out = ctypes.c_uint64()
        tot = ctypes.c_uint64()
        self._lib.oracle_range(self._h, lo, hi, ctypes.byref(out), None,
                               buf.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(tot))
        return buf[: min(cap, tot.value)].copy(), tot.value

    def _cube_checked(self, mask: int, r: int) -> int:
        if r == (1 << 64) - 1 and self.n - bin(mask & ((1 << self.n) - 1)).count("1") >= 64:
            raise ValueError("a subcube with 64 free variables has a count beyond 64 bits")
        return r

    def count_cube(self, mask: int, vals: int) -> int:
        """Models with the variables of ``mask`` fixed to the bits of ``vals``."""
        return self._cube_checked(mask, self._lib.oracle_count_cube(self._h, mask, vals))

    def count_cube_par(self, mask: int, vals: int, threads: int = 0) -> int:
        """count_cube with the subcube's points split across threads."""
        return self._cube_checked(mask, self._lib.oracle_count_cube_par(self._h, mask, vals, threads))

    def count_par(self, lo: int, hi: int, threads: int = 0) -> int:
        return self._lib.oracle_count_par(self._h, lo, hi, threads)


def cube_size(nf: int):
    """Points of a subcube with ``nf`` free variables (the loop bound both
    cube counters use), or None where the count need not fit 64 bits."""
    r = _load().oracle_cube_size(nf)
    return None if r == (1 << 64) - 1 else r


def max_threads() -> int:
    return _load().oracle_max_threads()
