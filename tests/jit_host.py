"""Compile the generated CUDA source of the specialised kernels as host C++
(test infrastructure).  The kernel body is straight-line integer code; the
few device builtins it uses get host stand-ins here, and one "thread" runs at
a time over all units (count mode: the lanes of one warp over every
(warp slice, unit) item).  Warp votes become per-thread votes (a thread skips
only levels whose partial conjunction is zero for itself, so counts and
tables are unchanged) and warp sums add over the lanes of a warp, run from
lane 31 down to lane 0.  This checks the emitter (folding, loops, stores) on
a machine without a GPU; it is not an evaluation path of the library.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1310_6978_b300", "csrc", "fbg_device.cuh")

PRELUDE = r'''
#include <cstdint>
#include <cstring>
#include "%s"
struct dim3_ { unsigned x, y, z; };
static dim3_ threadIdx;
#define __global__
#define __device__
#define __noinline__
#define __launch_bounds__(a, b)
#define __shared__ static
template <int LUT> static inline fbg_u32 fbg_lop3(fbg_u32 a, fbg_u32 b, fbg_u32 c) {
  fbg_u32 r = 0;
  for (int m = 0; m < 8; m++)
    if ((LUT >> m) & 1) r |= ((m & 4) ? a : ~a) & ((m & 2) ? b : ~b) & ((m & 1) ? c : ~c);
  return r;
}
static inline int __popc(fbg_u32 x) { return __builtin_popcount(x); }
static inline fbg_u32 fbg_madd(fbg_u32 a, fbg_u32 b, fbg_u32 one) { return a + b * one; }
static inline bool __any_sync(unsigned, bool p) { return p; }
static fbg_u64 g_warp_acc = 0;
static inline fbg_u64 fbg_warp_sum(fbg_u64 v) {
  g_warp_acc += v;
  if ((threadIdx.x & 31u) == 0u) { fbg_u64 r = g_warp_acc; g_warp_acc = 0; return r; }
  return v;
}
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) { auto o = *p; *p += v; return o; }
static inline unsigned long long atomicMin(unsigned long long* p, unsigned long long v) { auto o = *p; if (v < o) *p = v; return o; }
static inline fbg_u64 fbg_globaltimer() { return 0; }
static inline void __threadfence() {}
static inline void fbg_finish_count(const FbgLaunch& P, fbg_u64 total) {
  if (total) atomicAdd(P.acc, total);
  __threadfence();
  if (atomicAdd(P.done, 1ull) == (fbg_u64)P.nwarps - 1ull) {
    __threadfence();
    *P.out = atomicAdd(P.acc, 0ull);
    *P.acc = 0ull;
    *P.unit_ctr = 0ull;
    *P.done = 0ull;
  }
}
struct uint2 { fbg_u32 x, y; };
struct uint4 { fbg_u32 x, y, z, w; };
static inline uint2 make_uint2(fbg_u32 a, fbg_u32 b) { return uint2{a, b}; }
static inline uint4 make_uint4(fbg_u32 a, fbg_u32 b, fbg_u32 c, fbg_u32 d) { return uint4{a, b, c, d}; }
static fbg_u64 g_next = 0;
static inline fbg_u64 fbg_next_unit(const FbgLaunch& P, fbg_u64*) { return P.unit_begin + g_next++; }
static inline fbg_u64 fbg_next_units(const FbgLaunch& P, fbg_u64*, fbg_u64 c) { fbg_u64 u = P.unit_begin + g_next; g_next += c; return u; }
static inline fbg_u64 fbg_next_items_warp(const FbgLaunch&, fbg_u64 c) { fbg_u64 i = g_next; g_next += c; return i; }
'''

DRIVER = r'''
extern "C" int run(int mode, int block, unsigned long long nunits, unsigned long long* count, unsigned* table,
                   const unsigned* perm, unsigned long long nperm, int self_reset) {
  FbgLaunch P;
  std::memset(&P, 0, sizeof P);
  P.unit_perm = perm;
  P.nperm = nperm;
  unsigned long long acc = 0, done = 0, out = ~0ull;
  if (self_reset) { P.acc = &acc; P.done = &done; P.out = &out; P.nwarps = 1; }
  unsigned long long cnt = 0, ctr = 0;
  P.count = &cnt; P.unit_ctr = &ctr; P.table = table; P.unit_begin = 0; P.unit_end = nunits;
  P.chunk = nunits > 4 ? 3 : 1;   // ragged last chunk
  // count mode: one warp's lanes see every (warp slice, unit) item; table
  // mode: every thread of a block sees every unit
  for (int w = 0; w < (mode == 0 ? 1 : block / 32) || w == 0; w++) {
    for (int lane = 31; lane >= 0; lane--) {
      threadIdx.x = (unsigned)(w * 32 + lane);
      if ((int)threadIdx.x >= block) continue;
      g_next = 0;
      if (mode == 0) fbg_jit_count(P); else fbg_jit_table(P);
    }
  }
  *count = self_reset ? out : cnt;
  if (self_reset && (acc || done || cnt)) return 1;   // counters must be left zero
  return 0;
}
'''


def build_kernel(src: str, mode: int) -> ctypes.CDLL:
    kname = "fbg_jit_count" if mode == 0 else "fbg_jit_table"
    body = (PRELUDE % HDR) + src + DRIVER.replace("fbg_jit_count(P); else fbg_jit_table(P);",
                                                   f"{kname}(P); else {kname}(P);")
    h = hashlib.sha1(body.encode()).hexdigest()[:16]
    d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "jit_host")
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, f"k{h}.so")
    if not os.path.exists(so):
        cpp = os.path.join(d, f"k{h}.cpp")
        with open(cpp, "w") as f:
            f.write(body)
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-w", "-o", so + ".tmp", cpp])
        os.replace(so + ".tmp", so)
    lib = ctypes.CDLL(so)
    lib.run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_void_p,
                        ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_int]
    return lib


def run_count(src: str, block: int, nunits: int, perm=None, self_reset: bool = False) -> int:
    """Count; ``perm`` (uint32 array, entries unit << warp_bits | slice) is
    the list of items a launch hands out, in order (a scheduled launch, or
    only the live units); ``self_reset`` runs the protocol in which the last
    warp writes the total and zeroes the counters."""
    lib = build_kernel(src, 0)
    c = ctypes.c_ulonglong()
    pp, npp = None, 0
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.uint32)
        pp = perm.ctypes.data_as(ctypes.c_void_p) if len(perm) else ctypes.c_void_p(8)
        npp = len(perm)
    rc = lib.run(0, block, nunits, ctypes.byref(c), None, pp, npp, 1 if self_reset else 0)
    assert rc == 0, "counters not reset"
    return c.value


def run_table(src: str, block: int, nunits: int, nwords: int) -> np.ndarray:
    lib = build_kernel(src, 1)
    t = np.zeros(nwords, dtype=np.uint64)
    c = ctypes.c_ulonglong()
    lib.run(1, block, nunits, ctypes.byref(c), t.ctypes.data_as(ctypes.c_void_p), None, 0, 0)
    return t
