// interp_device.cuh -- device code of the bytecode interpreter (the kernels
// of interp.cu).  Evaluates the LUT bytecode of interp_format.h on 64-bit
// tiles: the bitwise evaluation of Sec. 2.3 with 64-bit blocks.  A block is
// one warp; each thread owns B / 32 tiles per innermost iteration (the
// layout's threads lane, lane + 32, ...), so every decoded instruction does
// the work of all of them (independent data paths per instruction); values
// live in shared memory (a thread's tiles of a slot in one 16-byte word, or
// one word per block for values equal in every tile) plus an accumulator
// register; loop levels run as an odometer; a level whose partial
// conjunction is zero for the whole warp skips its inner levels.
#pragma once

#include "fbg_device.cuh"
#include "interp_format.h"

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)

namespace fbg_interp {

constexpr int B = FBG_INTERP_BLOCK;          // tiles per block (the layout's threads), slot stride
constexpr int NT = FBG_INTERP_THREADS;       // threads per block
constexpr int NTILE = B / NT;                // tiles per thread
static_assert(NT == 32 && NTILE * NT == B, "one warp per block, B / 32 tiles per thread");
static_assert(NTILE == 2, "a thread's tiles of a slot are one 16-byte word");

// the tiles of a thread: tile k is the layout's thread lane + 32 k
struct Pair {
  fbg_u64 v[NTILE];
};

// lop3 needs its truth table as an immediate.  The (warp-uniform) LUT byte
// selects one of 256 code paths with one indirect branch (brx.idx over a
// table of 256 labels, label i holding the four lop3.b32 of both tiles with
// immediate i); a C++ switch over 256 cases is lowered to a tree of compares
// and branches instead.  Labels are local to the asm block's braces, so
// every inlined copy has its own.
#define FBG_LUT_CASE(v)                                                        \
  "L" #v ": lop3.b32 %0, %5, %9, %13, " #v ";\n\t"                           \
  "lop3.b32 %1, %6, %10, %14, " #v ";\n\t"                                   \
  "lop3.b32 %2, %7, %11, %15, " #v ";\n\t"                                   \
  "lop3.b32 %3, %8, %12, %16, " #v ";\n\t"                                   \
  "bra.uni LEND;\n"
#define FBG_LUT_ROW(h)                                                         \
  FBG_LUT_CASE(0x##h##0) FBG_LUT_CASE(0x##h##1) FBG_LUT_CASE(0x##h##2) FBG_LUT_CASE(0x##h##3) \
  FBG_LUT_CASE(0x##h##4) FBG_LUT_CASE(0x##h##5) FBG_LUT_CASE(0x##h##6) FBG_LUT_CASE(0x##h##7) \
  FBG_LUT_CASE(0x##h##8) FBG_LUT_CASE(0x##h##9) FBG_LUT_CASE(0x##h##A) FBG_LUT_CASE(0x##h##B) \
  FBG_LUT_CASE(0x##h##C) FBG_LUT_CASE(0x##h##D) FBG_LUT_CASE(0x##h##E) FBG_LUT_CASE(0x##h##F)
#define FBG_LUT_T(v) "L" #v
#define FBG_LUT_TROW(h)                                                        \
  FBG_LUT_T(0x##h##0) "," FBG_LUT_T(0x##h##1) "," FBG_LUT_T(0x##h##2) "," FBG_LUT_T(0x##h##3) "," \
  FBG_LUT_T(0x##h##4) "," FBG_LUT_T(0x##h##5) "," FBG_LUT_T(0x##h##6) "," FBG_LUT_T(0x##h##7) "," \
  FBG_LUT_T(0x##h##8) "," FBG_LUT_T(0x##h##9) "," FBG_LUT_T(0x##h##A) "," FBG_LUT_T(0x##h##B) "," \
  FBG_LUT_T(0x##h##C) "," FBG_LUT_T(0x##h##D) "," FBG_LUT_T(0x##h##E) "," FBG_LUT_T(0x##h##F)

__device__ __forceinline__ Pair lop3_dyn(unsigned lut, const Pair& a, const Pair& b, const Pair& c) {
  fbg_u32 d0, d1, d2, d3;
  asm volatile(
      "{\n\t"
      "LT: .branchtargets " FBG_LUT_TROW(0) "," FBG_LUT_TROW(1) "," FBG_LUT_TROW(2) "," FBG_LUT_TROW(3) ","
      FBG_LUT_TROW(4) "," FBG_LUT_TROW(5) "," FBG_LUT_TROW(6) "," FBG_LUT_TROW(7) "," FBG_LUT_TROW(8) ","
      FBG_LUT_TROW(9) "," FBG_LUT_TROW(A) "," FBG_LUT_TROW(B) "," FBG_LUT_TROW(C) "," FBG_LUT_TROW(D) ","
      FBG_LUT_TROW(E) "," FBG_LUT_TROW(F) ";\n\t"
      "brx.idx.uni %4, LT;\n"
      FBG_LUT_ROW(0) FBG_LUT_ROW(1) FBG_LUT_ROW(2) FBG_LUT_ROW(3) FBG_LUT_ROW(4) FBG_LUT_ROW(5) FBG_LUT_ROW(6)
      FBG_LUT_ROW(7) FBG_LUT_ROW(8) FBG_LUT_ROW(9) FBG_LUT_ROW(A) FBG_LUT_ROW(B) FBG_LUT_ROW(C) FBG_LUT_ROW(D)
      FBG_LUT_ROW(E) FBG_LUT_ROW(F)
      "LEND:\n\t}"
      : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3)
      : "r"(lut & 0xFFu), "r"((fbg_u32)a.v[0]), "r"((fbg_u32)(a.v[0] >> 32)), "r"((fbg_u32)a.v[1]),
        "r"((fbg_u32)(a.v[1] >> 32)), "r"((fbg_u32)b.v[0]), "r"((fbg_u32)(b.v[0] >> 32)), "r"((fbg_u32)b.v[1]),
        "r"((fbg_u32)(b.v[1] >> 32)), "r"((fbg_u32)c.v[0]), "r"((fbg_u32)(c.v[0] >> 32)), "r"((fbg_u32)c.v[1]),
        "r"((fbg_u32)(c.v[1] >> 32)));
  Pair d;
  d.v[0] = ((fbg_u64)d1 << 32) | d0;
  d.v[1] = ((fbg_u64)d3 << 32) | d2;
  return d;
}
#undef FBG_LUT_TROW
#undef FBG_LUT_T
#undef FBG_LUT_ROW
#undef FBG_LUT_CASE

struct Shared {
  FbgInterpProg prog;
  fbg_u64 svals[FBG_INTERP_MAX_SHARED];   // block slots: one word each, equal in every tile
  fbg_u64 unit;
  fbg_u64 item;
  // statistics launches (P.iters set): executions of each level by this
  // block, in units of 32 tiles (the block is one warp: lane 0 counts)
  fbg_u64 lev_iters[FBG_INTERP_MAX_LEVELS];
};

__device__ __forceinline__ void count_level(Shared& S, const FbgLaunch& P, int lv) {
  if (P.iters && (threadIdx.x & 31) == 0) S.lev_iters[lv] += NTILE;
}

struct Thread {
  fbg_u64* slots;       // this thread's tiles: tile k of slot s at slots[s * B + k] (16-byte aligned pair)
  Pair acc;
  fbg_u64 coords[NTILE];   // tile coordinates: bit positions >= 6 of j
};

__device__ __forceinline__ void init_thread(Thread& T, fbg_u64* dyn_slots) {
  T.slots = dyn_slots + threadIdx.x * NTILE;
#pragma unroll
  for (int k = 0; k < NTILE; k++) {
    T.acc.v[k] = 0;
    T.coords[k] = 0;
  }
}

__device__ __forceinline__ void set_thread_coords(Thread& T, fbg_u64 upper) {
#pragma unroll
  for (int k = 0; k < NTILE; k++) T.coords[k] = ((fbg_u64)(threadIdx.x + k * NT) << 6) | upper;
}

__device__ __forceinline__ Pair fetch(const Shared& S, const Thread& T, unsigned op) {
  Pair r;
  // tile slots (codes below FBG_OP_SHARED) are the most frequent operands:
  // one test, and 32-bit shared-memory offsets
  if (op < FBG_OP_SHARED) {
    // a thread's two tiles are adjacent: one 16-byte shared-memory load
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(T.slots + op * (unsigned)B);
    r.v[0] = v.x;
    r.v[1] = v.y;
    return r;
  }
  if (op == FBG_OP_ACC) return T.acc;
  if (op & FBG_OP_VAR) {
#pragma unroll
    for (int k = 0; k < NTILE; k++) r.v[k] = ((T.coords[k] >> (op & 63u)) & 1ull) ? ~0ull : 0ull;
    return r;
  }
  if (op & FBG_OP_CONST) {
    // the constant table stays in global memory (a few words, cached in L1):
    // no shared-memory copy per block, which leaves room for more blocks
    const fbg_u64 c = __ldg(S.prog.consts + (op & 0x3FFFu));
#pragma unroll
    for (int k = 0; k < NTILE; k++) r.v[k] = c;
    return r;
  }
  const fbg_u64 c = S.svals[op & 0xFFFu];   // a block slot
#pragma unroll
  for (int k = 0; k < NTILE; k++) r.v[k] = c;
  return r;
}

// instructions of one level; the next instruction word is loaded while the
// current one executes
__device__ __forceinline__ void exec_level(Shared& S, Thread& T, const FbgInterpLevel& L) {
  const fbg_u64* ins = S.prog.ins;
  unsigned i = L.ins_begin;
  if (i >= L.ins_end) return;
  fbg_u64 w = __ldg(ins + i);
  for (; i < L.ins_end; i++) {
    const fbg_u64 next = i + 1 < L.ins_end ? __ldg(ins + i + 1) : 0ull;
    const unsigned lut = (unsigned)(w & 0xFF), dst = (unsigned)((w >> 8) & 0xFF);
    const unsigned oa = (unsigned)((w >> 16) & 0xFFFF), ob = (unsigned)((w >> 32) & 0xFFFF), oc = (unsigned)(w >> 48);
    Pair d;
    if (((oa & ob & oc) & FBG_OP_VAR) && !(((oa | ob | oc) >> 6) & 0x1FFu)) {
      // all three operands are generator words of letters at positions >= 6
      // (no accumulator: its code has those bits set): each is all ones or
      // all zeros on a 64-bit tile, so the LUT is read at one index per tile
#pragma unroll
      for (int k = 0; k < NTILE; k++) {
        const fbg_u64 cw = T.coords[k];
        const unsigned idx = (unsigned)((((cw >> (oa & 63u)) & 1ull) << 2) | (((cw >> (ob & 63u)) & 1ull) << 1) |
                                        ((cw >> (oc & 63u)) & 1ull));
        d.v[k] = ((lut >> idx) & 1u) ? ~0ull : 0ull;
      }
    } else {
      const Pair a = fetch(S, T, oa);
      const Pair b = fetch(S, T, ob);
      const Pair c = fetch(S, T, oc);
      d = lop3_dyn(lut, a, b, c);
    }
    if (dst == FBG_DST_ACC) {
      T.acc = d;
    } else if (dst >= FBG_DST_SHARED) {
      // every lane computed the same word (the value is equal in all tiles);
      // the warp (the whole block) synchronises so that no lane overwrites a
      // block slot before every lane has read its previous value, and no lane
      // reads it before every lane has stored the new one
      __syncwarp();
      S.svals[dst - FBG_DST_SHARED] = d.v[0];
      __syncwarp();
    } else {
      *reinterpret_cast<ulonglong2*>(T.slots + dst * (unsigned)B) = make_ulonglong2(d.v[0], d.v[1]);
    }
    w = next;
  }
}

// MODE 0: count; 1: table (the table was zeroed before the launch); 2: enumerate
template <int MODE>
__device__ __forceinline__ bool level_alive(const Shared& S, const Thread& T, const FbgInterpLevel& L) {
  if (!L.has_acc) return true;
  const Pair v = fetch(S, T, L.acc_op);
  fbg_u64 any = 0;
#pragma unroll
  for (int k = 0; k < NTILE; k++) any |= v.v[k];
  const bool mine = any != 0ull;
  if (MODE == 2) return __syncthreads_or(mine) != 0;
  return __any_sync(FBG_FULL, mine);
}

__device__ __forceinline__ void load_prog(Shared& S, const FbgInterpProg* progs, unsigned p) {
  __syncthreads();
  if (threadIdx.x == 0) S.prog = progs[p];
  __syncthreads();
}

// inclusive prefix sum over the warp's lanes
__device__ __forceinline__ unsigned warp_incl(unsigned c) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(FBG_FULL, c, o);
    if (lane >= (unsigned)o) c += y;
  }
  return c;
}

template <int MODE>
__device__ void run_unit(Shared& S, Thread& T, fbg_u64 u, const FbgLaunch& P, fbg_u64& cnt) {
  const FbgInterpProg& G = S.prog;
  bool tvalid[NTILE];
#pragma unroll
  for (int k = 0; k < NTILE; k++) tvalid[k] = threadIdx.x + k * NT < G.tvalid;
  set_thread_coords(T, G.unit_bits ? (u << G.first_unit_pos) : 0ull);
  fbg_u64 base = 0;
  if (MODE == 2) {
    base = P.unit_offsets[u - P.unit_begin];
    if (base >= P.cap) return;   // every model of this unit lies past the cap
  }
  exec_level(S, T, G.lev[1]);
  count_level(S, P, 1);
  if (!level_alive<MODE>(S, T, G.lev[1])) return;
  // the loop nest as an odometer over the loop letters' bits, kept at their
  // own positions in lc (no per-level counter array, which would live in
  // local memory): a level's field is zero whenever the nest enters it
  fbg_u64 lc = 0;
  int lv = 2;
  const int nl = (int)G.nlevels;
  for (;;) {
    bool leaf = false;
    if (lv < nl) {
      const FbgInterpLevel& L = G.lev[lv];
      const fbg_u64 m = ((1ull << L.bits) - 1ull) << L.pos;
#pragma unroll
      for (int k = 0; k < NTILE; k++) T.coords[k] = (T.coords[k] & ~m) | (lc & m);
      exec_level(S, T, L);
      count_level(S, P, lv);
      bool alive = level_alive<MODE>(S, T, L);
      if (alive && lv + 1 < nl) {
        lv++;
        continue;
      }
      leaf = alive;
    } else {
      leaf = true;   // no loop levels: the unit level is innermost
    }
    if (leaf) {
      const Pair o = fetch(S, T, G.out_op);
      fbg_u64 word[NTILE];
#pragma unroll
      for (int k = 0; k < NTILE; k++) word[k] = tvalid[k] ? (o.v[k] & G.vmask) : 0ull;
      if (MODE == 0) {
#pragma unroll
        for (int k = 0; k < NTILE; k++) cnt += (fbg_u64)__popcll(word[k]);
      } else if (MODE == 1) {
#pragma unroll
        for (int k = 0; k < NTILE; k++)
          if (tvalid[k]) reinterpret_cast<fbg_u64*>(P.table)[(T.coords[k] >> 6) - P.table_word0] = word[k];
      } else {
        // ordered compaction: tiles ascend with lane + 32 k, so all tiles 0
        // of the warp precede all tiles 1
        fbg_u64 off = base;
#pragma unroll
        for (int k = 0; k < NTILE; k++) {
          const unsigned c = (unsigned)__popcll(word[k]);
          const unsigned incl = warp_incl(c);
          const unsigned total = __shfl_sync(FBG_FULL, incl, 31);
          fbg_u64 o2 = off + incl - c;
          fbg_u64 wd = word[k];
          while (wd) {
            int b = __ffsll((long long)wd) - 1;
            wd &= wd - 1;
            if (o2 < P.cap) P.models[o2] = T.coords[k] | (fbg_u64)b;
            o2++;
          }
          off += total;
        }
        base = off;
      }
    }
    if (lv < 2 || nl <= 2) break;
    // odometer advance: add one at the current level; a level that wraps
    // to zero carries into the level above
    for (;;) {
      const FbgInterpLevel& L = G.lev[lv];
      const fbg_u64 m = ((1ull << L.bits) - 1ull) << L.pos;
      const fbg_u64 f = ((lc & m) + (1ull << L.pos)) & m;
      lc = (lc & ~m) | f;
      if (f != 0ull || --lv < 2) break;
    }
    if (lv < 2) break;
  }
}

// one work item (program, unit range) of a count / table / enumerate pass
template <int MODE>
__device__ __forceinline__ void process_item(Shared& S, Thread& T, const FbgInterpProg* progs, const FbgWorkItem& W,
                                             unsigned& cur, bool& alive0, const FbgLaunch& P, fbg_u64& cnt) {
  if (W.prog != cur) {
    load_prog(S, progs, W.prog);
    cur = W.prog;
    set_thread_coords(T, 0ull);
    exec_level(S, T, S.prog.lev[0]);
    count_level(S, P, 0);
    alive0 = level_alive<MODE>(S, T, S.prog.lev[0]);
  }
  if (alive0)
    for (fbg_u64 u = W.unit_begin; u < W.unit_end; u++) run_unit<MODE>(S, T, u, P, cnt);
}

}  // namespace fbg_interp

#endif  // __CUDACC__ || __CUDACC_RTC__
