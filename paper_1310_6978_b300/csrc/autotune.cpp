// autotune.cpp -- per-program choice of the specialised kernel's shape.
//
// The layout knobs -- 32-bit registers per thread tile (words per thread),
// warps per block, minimum resident blocks (register budget), bits per loop
// level (which also sets the unrolled innermost depth) and unit bits -- are
// searched coordinate by coordinate from the current setting: each knob's
// alternatives are compiled (NVRTC) and timed with CUDA events on the
// caller's stream, the fastest is kept, and the program is left configured
// with the best shape found.  Counts are timed after fbg_schedule_units, so
// each shape is timed with its own longest-first unit order, and the
// program keeps the order of the chosen shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fbg.h"
#include "program.hpp"

using namespace fbg;

namespace {

struct Knob {
  int option;
  std::vector<int64_t> values;
};

double time_once(fbg_program* p, int mode, cudaStream_t st, void* table, size_t nwords, int reps, fbg_status* err) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  unsigned long long* dcount = nullptr;
  *err = FBG_OK;
  double best = 1e30;
  // first call compiles and warms up; counts are timed in their measured order
  uint64_t c = 0;
  *err = mode == 0 ? fbg_count(p, st, &c) : fbg_truth_table(p, st, (uint64_t*)table, nwords);
  if (*err == FBG_OK && mode == 0) *err = fbg_schedule_units(p, st);
  if (*err == FBG_OK && cudaStreamSynchronize(st) != cudaSuccess) *err = FBG_ECUDA;
  if (*err == FBG_OK && mode == 0 && cudaMalloc(&dcount, 8) != cudaSuccess) *err = FBG_ENOMEM;
  // reps rounds of kLaunches launches enqueued back to back (the host runs
  // ahead, so the events time the GPU); the best round's mean per launch
  const int kLaunches = 8;
  for (int r = 0; r < reps && *err == FBG_OK; r++) {
    cudaEventRecord(e0, st);
    for (int l = 0; l < kLaunches && *err == FBG_OK; l++)
      *err = mode == 0 ? fbg_count_async(p, st, (uint64_t*)dcount) : fbg_truth_table(p, st, (uint64_t*)table, nwords);
    cudaEventRecord(e1, st);
    if (*err != FBG_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *err = FBG_ECUDA;
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, (double)ms / kLaunches);
  }
  if (dcount) cudaFree(dcount);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

extern "C" fbg_status fbg_autotune(fbg_program* p, void* stream, int mode, int reps, fbg_tune_result* out) {
  if (!p || !out || (mode != 0 && mode != 1)) return set_error(FBG_EINVAL, "bad argument");
  if (mode == 1 && p->n > 34) return set_error(FBG_ETOOBIG, "table tuning needs n <= 34");
  cudaStream_t st = (cudaStream_t)stream;
  if (reps <= 0) reps = 3;
  int64_t saved_engine = p->opt_engine;
  p->opt_engine = FBG_ENGINE_JIT;
  void* table = nullptr;
  size_t nwords = p->n <= 6 ? 1 : (size_t)1 << (p->n - 6);
  if (mode == 1) {
    cudaError_t e = cudaMalloc(&table, nwords * 8);
    if (e != cudaSuccess) {
      p->opt_engine = saved_engine;
      return cuda_error(e, "autotune table buffer");
    }
  }
  const std::vector<Knob> knobs = {
      {FBG_OPT_LOOP_LEVEL_BITS, {2, 3, 4, 5}},
      {FBG_OPT_REGS_LOG2, {1, 2, 3}},
      {FBG_OPT_MIN_BLOCKS, {1, 2, 3}},
      {FBG_OPT_WARPS_LOG2, {2, 3, 4}},
      {FBG_OPT_UNIT_BITS, {10, 12, 13, 14}},
      {FBG_OPT_INNER_BITS, {0, 1, 3, 4}},
      {FBG_OPT_POPC_COST, {0, 2, 4, 8}},
      {FBG_OPT_ORDER_SEED, {0, 1, 2, 3, 4, 5, 6, 7}},
  };
  auto get = [&](int opt) -> int64_t {
    switch (opt) {
      case FBG_OPT_LOOP_LEVEL_BITS: return p->opt_loop_level_bits;
      case FBG_OPT_REGS_LOG2: return p->opt_regs_log2;
      case FBG_OPT_MIN_BLOCKS: return p->opt_min_blocks;
      case FBG_OPT_WARPS_LOG2: return p->opt_warps_log2;
      case FBG_OPT_INNER_BITS: return p->opt_inner_bits;
      case FBG_OPT_POPC_COST: return p->opt_popc_cost;
      case FBG_OPT_ORDER_SEED: return p->opt_order_seed;
      default: return p->opt_unit_bits;
    }
  };
  fbg_status err = FBG_OK;
  double best = time_once(p, mode, st, table, nwords, reps, &err);
  int trials = 1;
  if (err != FBG_OK) {
    if (table) cudaFree(table);
    p->opt_engine = saved_engine;
    return err;
  }
  for (const Knob& k : knobs) {
    if (mode != 0 && (k.option == FBG_OPT_ORDER_SEED || k.option == FBG_OPT_POPC_COST)) continue;   // count-only knobs
    int64_t keep = get(k.option);
    for (int64_t v : k.values) {
      if (v == keep) continue;
      if (fbg_set_option(p, k.option, v) != FBG_OK) continue;
      double t = time_once(p, mode, st, table, nwords, reps, &err);
      trials++;
      if (err == FBG_OK && t < best) {
        best = t;
        keep = v;
      }
    }
    fbg_set_option(p, k.option, keep);
  }
  // leave the program built with the chosen shape
  double t = time_once(p, mode, st, table, nwords, 1, &err);
  (void)t;
  if (table) cudaFree(table);
  p->opt_engine = saved_engine;
  out->best_ms = best;
  out->trials = trials;
  out->regs_log2 = (int)p->opt_regs_log2;
  out->warps_log2 = (int)p->opt_warps_log2;
  out->min_blocks = (int)p->opt_min_blocks;
  out->loop_level_bits = (int)p->opt_loop_level_bits;
  out->unit_bits = (int)p->opt_unit_bits;
  out->inner_bits = (int)p->opt_inner_bits;
  out->popc_cost = (int)p->opt_popc_cost;
  out->order_seed = (int)p->opt_order_seed;
  return err;
}
