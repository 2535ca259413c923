// fbg_device.cuh -- definitions shared by the interpreter kernels (nvcc) and
// the NVRTC-specialised kernels (this file is embedded as text and prepended
// to every generated source).  No includes: NVRTC compiles it standalone.
#pragma once

typedef unsigned int fbg_u32;
typedef unsigned long long fbg_u64;

// One launch of a count / table / enumerate pass over the units
// [unit_begin, unit_end) of one program.
struct FbgLaunch {
  fbg_u64* count;          // += number of models (device u64), may be null
  fbg_u64* unit_counts;    // per-unit model counts (index u - unit_begin), may be null
  fbg_u32* table;          // truth table as 32-bit words (table mode)
  fbg_u64* models;         // model list (enumerate mode)
  const fbg_u64* unit_offsets;   // enumerate: exclusive prefix of unit counts
  fbg_u64* unit_ctr;       // dynamic unit counter, zero before the launch
  fbg_u64* iters;          // optional: innermost-level iterations executed (+=)
  fbg_u64 cap;             // enumerate: capacity of `models`
  fbg_u64 unit_begin, unit_end;
  fbg_u64 chunk;           // units fetched per counter increment (0 = 1)
  fbg_u64* unit_trace;     // optional diagnostics (count mode): per unit (index u - unit_begin)
                           // [2u] += warp-nanoseconds spent, [2u+1] = min start time (ns)
  fbg_u64* item_trace;     // optional (count mode): nanoseconds of item (unit u, warp slice w)
                           // at index (u - unit_begin) * slices + w
  const fbg_u32* unit_perm;  // optional (count mode, full range): the items handed out, in order,
                             // each entry u << warp_bits | w (< 2^24; units with no models may be
                             // left out), plus s << 28 | q << 24: piece q of 2^s of the values of
                             // the first loop level (s = 0: the whole item)
  fbg_u64 nperm;             // number of entries of unit_perm
  fbg_u64* acc;            // self-resetting count (count mode, when done is set): running sum,
  fbg_u64* done;           //   warps finished, the destination of the total, warps in the grid;
  fbg_u64* out;            //   acc, done and unit_ctr are zero before the launch and after it
  fbg_u32 nwarps;
  fbg_u64 table_word0;     // table mode: 64-bit word index of the first word of `table` (a slice
                           // of the units [unit_begin, unit_end); 0 for a whole table)
};

#define FBG_FULL 0xffffffffu

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)

template <int LUT>
__device__ __forceinline__ fbg_u32 fbg_lop3(fbg_u32 a, fbg_u32 b, fbg_u32 c) {
  fbg_u32 d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

__device__ __forceinline__ fbg_u64 fbg_warp_sum(fbg_u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FBG_FULL, v, o);
  return v;
}

// generator word of a non-constant bit position: all ones where the bit is 1
__device__ __forceinline__ fbg_u32 fbg_genword(fbg_u64 coord, int bit) {
  return 0u - (fbg_u32)((coord >> bit) & 1ull);
}

// fetch the next unit for the whole block (dynamic, atomic counter)
__device__ __forceinline__ fbg_u64 fbg_next_unit(const FbgLaunch& P, fbg_u64* s_unit) {
  if (threadIdx.x == 0) *s_unit = P.unit_begin + atomicAdd(P.unit_ctr, 1ull);
  __syncthreads();
  fbg_u64 u = *s_unit;
  __syncthreads();
  return u;
}

// fetch the next `chunk` units for the whole block
// a + b * one as an integer multiply-add: with `one` a runtime 1 the
// compiler cannot fold, the add issues on the FMA pipe instead of the ALU
// pipe that the lop3 work saturates
__device__ __forceinline__ fbg_u32 fbg_madd(fbg_u32 a, fbg_u32 b, fbg_u32 one) {
  fbg_u32 d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(b), "r"(one), "r"(a));
  return d;
}

// the global nanosecond timer (diagnostics only)
__device__ __forceinline__ fbg_u64 fbg_globaltimer() {
  fbg_u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Self-resetting count, which needs no memset before a launch: every warp
// adds its total to *acc and then counts itself done; the warp that finishes
// last writes the sum to *out and zeroes acc, done and the item counter for
// the next launch.  No warp waits for another (call from one lane per warp).
__device__ __forceinline__ void fbg_finish_count(const FbgLaunch& P, fbg_u64 total) {
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

// The next chunk of work items for the calling warp: lane 0 draws from the
// counter and the other lanes receive the index; no block barrier, so a warp
// never waits for the other warps of its block.
__device__ __forceinline__ fbg_u64 fbg_next_items_warp(const FbgLaunch& P, fbg_u64 chunk) {
  fbg_u64 i = 0;
  if ((threadIdx.x & 31u) == 0u) i = atomicAdd(P.unit_ctr, chunk);
  return __shfl_sync(0xffffffffu, i, 0);
}

__device__ __forceinline__ fbg_u64 fbg_next_units(const FbgLaunch& P, fbg_u64* s_unit, fbg_u64 chunk) {
  if (threadIdx.x == 0) *s_unit = P.unit_begin + atomicAdd(P.unit_ctr, chunk);
  __syncthreads();
  fbg_u64 u = *s_unit;
  __syncthreads();
  return u;
}

#endif  // __CUDACC__ || __CUDACC_RTC__
