// interp_device.cuh -- device code of the bytecode interpreter, shared by the
// nvcc-compiled kernels (interp.cu) and the NVRTC-compiled batch kernel that
// mixes interpreted and specialised programs.  Evaluates the LUT bytecode of
// interp_format.h on 64-bit tiles: the bitwise evaluation of Sec. 2.3 with
// 64-bit blocks.  Each thread owns one tile per innermost iteration; values
// live in a per-thread column of shared memory plus an accumulator register;
// loop levels run as an odometer; a level whose partial conjunction is zero
// for a whole warp (for model lists: the whole block) skips its inner levels.
#pragma once

#include "fbg_device.cuh"
#include "interp_format.h"

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)

namespace fbg_interp {

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
  return T.slots[(unsigned long long)op * B];
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
    else T.slots[(unsigned long long)dst * B] = d;
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

// one work item (program, unit range) of a count / table / enumerate pass
template <int MODE>
__device__ __forceinline__ void process_item(Shared& S, Thread& T, const FbgInterpProg* progs, const FbgWorkItem& W,
                                             unsigned& cur, bool& alive0, const FbgLaunch& P, fbg_u64& cnt,
                                             fbg_u64& iters) {
  if (W.prog != cur) {
    load_prog(S, progs, W.prog);
    cur = W.prog;
    T.coords = (fbg_u64)threadIdx.x << 6;
    exec_level(S, T, S.prog.lev[0]);
    alive0 = level_alive<MODE>(S, T, S.prog.lev[0]);
  }
  if (alive0)
    for (fbg_u64 u = W.unit_begin; u < W.unit_end; u++) run_unit<MODE>(S, T, u, P, cnt, iters);
}

}  // namespace fbg_interp

#endif  // __CUDACC__ || __CUDACC_RTC__
