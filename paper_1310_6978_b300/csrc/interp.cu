// interp.cu -- generic bytecode interpreter kernels (sm_103a).
//
// Evaluates any compiled program without a JIT: the formula is a list of
// 3-input LUT instructions (interp_format.h) on 64-bit tile words, i.e. the
// bitwise evaluation d_j = t(b_1j..b_nj) of Sec. 2.3 with 64-bit blocks.
// Each thread owns one 64-bit tile per innermost iteration; the generator
// words of bits >= 6 are all-ones/all-zeros words derived from the tile's
// coordinates, bits 0..5 are the constant masks folded into the program.
// Values live in a per-thread column of shared memory (slot s of thread t at
// slots[s*BLOCK+t]) plus one accumulator register.  Loop levels run as an
// odometer; a level whose partial conjunction is zero for a whole warp (for
// enumeration: the whole block) skips its inner levels.
//
// One kernel serves single programs and the persistent batch: blocks pull
// work items (program, unit range) from a device counter.
#include <cuda_runtime.h>

#include "fbg_device.cuh"
#include "interp_format.h"
#include "kernels.hpp"

namespace fbg {

template <int LUT>
__device__ __forceinline__ fbg_u64 lop3_pair(fbg_u64 a, fbg_u64 b, fbg_u64 c) {
  fbg_u32 lo = fbg_lop3<LUT>((fbg_u32)a, (fbg_u32)b, (fbg_u32)c);
  fbg_u32 hi = fbg_lop3<LUT>((fbg_u32)(a >> 32), (fbg_u32)(b >> 32), (fbg_u32)(c >> 32));
  return ((fbg_u64)hi << 32) | lo;
}

// lop3 needs its truth table as an immediate: dispatch on the (warp-uniform) LUT
__device__ __forceinline__ fbg_u64 lop3_dyn(unsigned lut, fbg_u64 a, fbg_u64 b, fbg_u64 c) {
  switch (lut) {
#define FBG_C(x) \
  case (x): return lop3_pair<(x)>(a, b, c);
#define FBG_C4(x) FBG_C(x) FBG_C((x) + 1) FBG_C((x) + 2) FBG_C((x) + 3)
#define FBG_C16(x) FBG_C4(x) FBG_C4((x) + 4) FBG_C4((x) + 8) FBG_C4((x) + 12)
#define FBG_C64(x) FBG_C16(x) FBG_C16((x) + 16) FBG_C16((x) + 32) FBG_C16((x) + 48)
    FBG_C64(0) FBG_C64(64) FBG_C64(128) FBG_C64(192)
#undef FBG_C64
#undef FBG_C16
#undef FBG_C4
#undef FBG_C
  }
  return 0;
}

namespace {

constexpr int B = FBG_INTERP_BLOCK;
constexpr int MAX_CONST_SMEM = FBG_INTERP_MAX_CONSTS;

struct Shared {
  FbgInterpProg prog;
  fbg_u64 consts[MAX_CONST_SMEM];
  fbg_u64 unit;
  fbg_u64 item;
  fbg_u32 warp_tot[B / 32];
};

struct Thread {
  fbg_u64* slots;       // this thread's column
  fbg_u64 acc;
  fbg_u64 coords;       // tile coordinates: bit positions >= 6 of j
};

__device__ __forceinline__ fbg_u64 fetch(const Shared& S, const Thread& T, unsigned op) {
  if (op == FBG_OP_ACC) return T.acc;
  if (op & FBG_OP_VAR) return ((T.coords >> (op & 63u)) & 1ull) ? ~0ull : 0ull;
  if (op & FBG_OP_CONST) return S.consts[op & 0x3FFFu];
  return T.slots[(size_t)op * B];
}

__device__ __forceinline__ void exec_level(const Shared& S, Thread& T, const FbgInterpLevel& L) {
  const fbg_u64* ins = S.prog.ins;
  for (unsigned i = L.ins_begin; i < L.ins_end; i++) {
    fbg_u64 w = __ldg(ins + i);
    unsigned lut = (unsigned)(w & 0xFF), dst = (unsigned)((w >> 8) & 0xFF);
    fbg_u64 a = fetch(S, T, (unsigned)((w >> 16) & 0xFFFF));
    fbg_u64 b = fetch(S, T, (unsigned)((w >> 32) & 0xFFFF));
    fbg_u64 c = fetch(S, T, (unsigned)(w >> 48));
    fbg_u64 d = lop3_dyn(lut, a, b, c);
    if (dst == FBG_DST_ACC) T.acc = d;
    else T.slots[(size_t)dst * B] = d;
  }
}

// MODE 0: count; 1: table (the table was zeroed before the launch); 2: enumerate
template <int MODE>
__device__ __forceinline__ bool level_alive(const Shared& S, const Thread& T, const FbgInterpLevel& L) {
  if (!L.has_acc) return true;
  bool mine = fetch(S, T, L.acc_op) != 0ull;
  if (MODE == 2) return __syncthreads_or(mine) != 0;
  return __any_sync(FBG_FULL, mine);
}

__device__ __forceinline__ void load_prog(Shared& S, const FbgInterpProg* progs, unsigned p) {
  __syncthreads();
  if (threadIdx.x == 0) S.prog = progs[p];
  __syncthreads();
  for (unsigned i = threadIdx.x; i < S.prog.nconst && i < MAX_CONST_SMEM; i += B) S.consts[i] = S.prog.consts[i];
  __syncthreads();
}

template <int MODE>
__device__ void run_unit(Shared& S, Thread& T, fbg_u64 u, const FbgLaunch& P, fbg_u64& cnt, fbg_u64& iters) {
  const FbgInterpProg& G = S.prog;
  const unsigned tb = threadIdx.x;
  const bool tvalid = tb < G.tvalid;
  T.coords = ((fbg_u64)tb << 6) | (G.unit_bits ? (u << G.first_unit_pos) : 0ull);
  fbg_u64 base = 0;
  if (MODE == 2) base = P.unit_offsets[u - P.unit_begin];
  exec_level(S, T, G.lev[1]);
  if (!level_alive<MODE>(S, T, G.lev[1])) return;
  unsigned it[FBG_INTERP_MAX_LEVELS];
  int lv = 2;
  const int nl = (int)G.nlevels;
  if (nl > 2) it[2] = 0;
  for (;;) {
    bool leaf = false;
    if (lv < nl) {
      const FbgInterpLevel& L = G.lev[lv];
      fbg_u64 m = ((1ull << L.bits) - 1ull) << L.pos;
      T.coords = (T.coords & ~m) | ((fbg_u64)it[lv] << L.pos);
      exec_level(S, T, L);
      bool alive = level_alive<MODE>(S, T, L);
      if (alive && lv + 1 < nl) {
        lv++;
        it[lv] = 0;
        continue;
      }
      leaf = alive;
    } else {
      leaf = true;   // no loop levels: the unit level is innermost
    }
    if (leaf) {
      fbg_u64 word = tvalid ? (fetch(S, T, G.out_op) & G.vmask) : 0ull;
      if (MODE == 0) {
        cnt += (fbg_u64)__popcll(word);
      } else if (MODE == 1) {
        if (tvalid) reinterpret_cast<fbg_u64*>(P.table)[T.coords >> 6] = word;
      } else {
        // ordered compaction across the block: tiles ascend with threadIdx
        unsigned c = (unsigned)__popcll(word);
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          unsigned y = __shfl_up_sync(FBG_FULL, incl, o);
          if ((tb & 31) >= (unsigned)o) incl += y;
        }
        if ((tb & 31) == 31) S.warp_tot[tb >> 5] = incl;
        __syncthreads();
        unsigned before = 0, total = 0;
        for (int w = 0; w < B / 32; w++) {
          if (w < (int)(tb >> 5)) before += S.warp_tot[w];
          total += S.warp_tot[w];
        }
        __syncthreads();
        fbg_u64 off = base + before + incl - c;
        while (word) {
          int b = __ffsll((long long)word) - 1;
          word &= word - 1;
          if (off < P.cap) P.models[off] = T.coords | (fbg_u64)b;
          off++;
        }
        base += total;
      }
      if ((tb & 31) == 0) iters++;
    }
    if (lv < 2 || nl <= 2) break;
    // odometer advance
    while (lv >= 2 && ++it[lv] == (1u << G.lev[lv].bits)) lv--;
    if (lv < 2) break;
  }
}

template <int MODE>
__global__ void __launch_bounds__(B) interp_kernel(const FbgInterpProg* __restrict__ progs,
                                                   const FbgWorkItem* __restrict__ items, fbg_u64 nitems,
                                                   fbg_u64* item_ctr, fbg_u64* prog_counts, fbg_u64* item_counts,
                                                   FbgLaunch P) {
  extern __shared__ fbg_u64 dyn_slots[];
  __shared__ Shared S;
  Thread T;
  T.slots = dyn_slots + threadIdx.x;
  T.acc = 0;
  unsigned cur = 0xFFFFFFFFu;
  bool alive0 = true;
  fbg_u64 iters = 0;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(item_ctr, 1ull);
    __syncthreads();
    fbg_u64 item = S.item;
    __syncthreads();
    if (item >= nitems) break;
    FbgWorkItem W = items[item];
    if (W.prog != cur) {
      load_prog(S, progs, W.prog);
      cur = W.prog;
      T.coords = (fbg_u64)threadIdx.x << 6;
      exec_level(S, T, S.prog.lev[0]);
      alive0 = level_alive<MODE>(S, T, S.prog.lev[0]);
    }
    fbg_u64 cnt = 0;
    if (alive0)
      for (fbg_u64 u = W.unit_begin; u < W.unit_end; u++) run_unit<MODE>(S, T, u, P, cnt, iters);
    if (MODE == 0) {
      cnt = fbg_warp_sum(cnt);
      if ((threadIdx.x & 31) == 0 && cnt) {
        if (prog_counts) atomicAdd(prog_counts + W.prog, cnt);
        if (item_counts) atomicAdd(item_counts + item, cnt);
      }
    }
  }
  if (P.iters && (threadIdx.x & 31) == 0 && iters) atomicAdd(P.iters, iters);
}

// exclusive prefix sum of n u64 values, one block; total -> *total
__global__ void scan_kernel(const fbg_u64* in, fbg_u64* out, fbg_u64 n, fbg_u64* total) {
  __shared__ fbg_u64 part[1024];
  const unsigned t = threadIdx.x;
  fbg_u64 per = (n + 1023) / 1024;
  fbg_u64 lo = t * per, hi = lo + per < n ? lo + per : n;
  fbg_u64 s = 0;
  for (fbg_u64 i = lo; i < hi; i++) s += in[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    fbg_u64 run = 0;
    for (int i = 0; i < 1024; i++) {
      fbg_u64 v = part[i];
      part[i] = run;
      run += v;
    }
    if (total) *total = run;
  }
  __syncthreads();
  fbg_u64 run = part[t];
  for (fbg_u64 i = lo; i < hi; i++) {
    fbg_u64 v = in[i];
    out[i] = run;
    run += v;
  }
}

}  // namespace

size_t interp_smem_bytes(unsigned nslots) { return (size_t)nslots * B * sizeof(fbg_u64); }

// the dynamic shared memory limit is raised only when a larger size is needed,
// so launches (also inside stream capture) do not call cudaFuncSetAttribute
static cudaError_t ensure_smem(int mode, size_t smem) {
  static size_t set_to[3] = {0, 0, 0};
  if (smem <= set_to[mode]) return cudaSuccess;
  cudaError_t e;
  if (mode == 0) e = cudaFuncSetAttribute(interp_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (mode == 1) e = cudaFuncSetAttribute(interp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else e = cudaFuncSetAttribute(interp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set_to[mode] = smem;
  return e;
}

cudaError_t launch_interp(int mode, const FbgInterpProg* progs, const FbgWorkItem* items, unsigned long long nitems,
                          unsigned long long* item_ctr, unsigned long long* prog_counts,
                          unsigned long long* item_counts, const FbgLaunch& P, unsigned nslots, int grid,
                          cudaStream_t stream) {
  size_t smem = interp_smem_bytes(nslots);
  cudaError_t e = ensure_smem(mode, smem);
  if (e != cudaSuccess) return e;
  if (mode == 0)
    interp_kernel<0><<<grid, B, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, item_counts, P);
  else if (mode == 1)
    interp_kernel<1><<<grid, B, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, item_counts, P);
  else
    interp_kernel<2><<<grid, B, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, item_counts, P);
  return cudaGetLastError();
}

cudaError_t launch_scan(const unsigned long long* in, unsigned long long* out, unsigned long long n,
                        unsigned long long* total, cudaStream_t stream) {
  scan_kernel<<<1, 1024, 0, stream>>>(in, out, n, total);
  return cudaGetLastError();
}

int interp_blocks_per_sm(int mode, unsigned nslots) {
  int nb = 0;
  size_t smem = interp_smem_bytes(nslots);
  if (ensure_smem(mode, smem) != cudaSuccess) return 0;
  if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<0>, B, smem);
  else if (mode == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<1>, B, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<2>, B, smem);
  return nb;
}

}  // namespace fbg
