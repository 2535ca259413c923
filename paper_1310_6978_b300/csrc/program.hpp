// program.hpp -- the compiled program behind the opaque fbg_program handle.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "emit.hpp"
#include "fbg.h"
#include "fbg_internal.hpp"

namespace fbg {

struct InterpBuild {
  bool valid = false;
  LutProgram lp;
  InterpCode code;
  FbgInterpProg* d_prog = nullptr;
  unsigned long long* d_ins = nullptr;
  unsigned long long* d_consts = nullptr;
  FbgWorkItem* d_items = nullptr;
  uint64_t nitems = 0, nunits = 0, units_per_item = 1;
  int grid = 1;
  // the units that can have models, ascending (null = all); units on which a
  // conjunct over unit and warp letters is false are left out.  Shared with
  // the host build cache, not copied per program
  std::shared_ptr<const std::vector<uint32_t>> live;
  uint64_t live_units() const { return live ? (uint64_t)live->size() : nunits; }
  uint64_t unit_at(uint64_t i) const { return live ? (uint64_t)(*live)[(size_t)i] : i; }
  // work items over the live units with positions [lo, hi): runs of
  // consecutive units, at most max_units each
  void append_items(std::vector<FbgWorkItem>& out, unsigned prog, uint64_t lo, uint64_t hi,
                    uint64_t max_units) const {
    uint64_t i = lo;
    while (i < hi) {
      const uint64_t u0 = unit_at(i);
      uint64_t len = 1;
      while (i + len < hi && len < max_units && unit_at(i + len) == u0 + len) len++;
      out.push_back(FbgWorkItem{prog, 0u, u0, u0 + len});
      i += len;
    }
  }
  // descriptor, bytecode, constants and items share one device allocation
  // (d_prog is its start); a build from the stream-ordered pool is freed in
  // the order of free_stream, without waiting for the device
  bool pooled = false;
  cudaStream_t free_stream = nullptr;
  void free_device() {
    if (d_prog) {
      if (pooled) cudaFreeAsync(d_prog, free_stream);
      else cudaFree(d_prog);
    }
    pooled = false;
    d_prog = nullptr;
    d_ins = d_consts = nullptr;
    d_items = nullptr;
  }
};

struct JitBuild {
  bool valid = false;
  LutProgram lp;
  std::string src, log;
  std::vector<long long> ops;    // lane-varying lop3.b32 per thread per level execution (after folding)
  std::vector<long long> uops;   // warp-uniform lop3 per warp per level execution
  int unrolled_level = -1;       // loop level emitted unrolled (one execution = all iterations)
  cudaKernel_t kern = nullptr;   // owned by the process-wide JIT cache
  int block = 256, grid = 1;
  uint64_t nunits = 1;
  unsigned* d_perm = nullptr;    // items of full-range counts, in order, or null (all, natural order)
  uint64_t nperm = 0;
  std::shared_ptr<void> perm_owner;   // set when d_perm is the shared list of a cached build
  std::vector<uint8_t> alive;    // per (unit, warp slice) item: 0 = no models, empty = all live
  void free_device() {
    if (d_perm && !perm_owner) cudaFree(d_perm);
    perm_owner.reset();
    d_perm = nullptr;
    nperm = 0;
  }
};

fbg_status set_error(fbg_status s, const std::string& m);
fbg_status cuda_error(cudaError_t e, const char* where);
int device_sms();

}  // namespace fbg

namespace fbg {
// The parsed and grounded theory of one (text, domain size): immutable once
// built and shared by every program compiled from the same text
// (compile_cached keeps recent ones).
struct Compiled {
  Theory th;
  Grounded g;
};
std::shared_ptr<const Compiled> compile_cached(const std::string& text, int k);   // throws CompileError
}  // namespace fbg

struct fbg_program {
  std::string text;
  int k = 1;
  int n = 0;
  std::shared_ptr<const fbg::Compiled> compiled;
  const fbg::Theory* th = nullptr;      // = &compiled->th
  const fbg::Grounded* g = nullptr;     // = &compiled->g
  // options (fbg_set_option)
  int64_t opt_engine = FBG_ENGINE_AUTO, opt_prune = 1, opt_regs_log2 = 2, opt_warps_log2 = 3, opt_unit_bits = 13,
          opt_loop_level_bits = 0, opt_search = 1, opt_min_blocks = 2, opt_stats = 0, opt_inner_bits = 0,
          opt_split_items = 0, opt_popc_cost = 4, opt_order_seed = 0;
  fbg::InterpBuild ib[2];   // [0] count layout, [1] identity layout (tables, model lists)
  fbg::JitBuild jb[3];      // [0] count kernel, [1] truth-table kernel, [2] enumerate kernel
  unsigned long long* d_scratch = nullptr;
  bool scratch_clean = false;   // counters of self-resetting count launches are zero
  // when set (by the server), interpreter builds come from the stream-ordered
  // pool: allocated and uploaded on alloc_stream, freed on free_stream
  cudaStream_t alloc_stream = nullptr, free_stream = nullptr;
  size_t scratch_words = 0;
  fbg_exec_stats last{};
  // wall time (s) in kernel builds and in fbg_count outside builds (fbg_debug_host_times)
  double t_build = 0, t_count = 0;
  std::string jit_log;

  void invalidate() {
    for (auto& b : ib) {
      b.free_device();
      b = fbg::InterpBuild{};
    }
    for (auto& b : jb) {
      b.free_device();
      b = fbg::JitBuild{};
    }
  }
  ~fbg_program() {
    for (auto& b : ib) b.free_device();
    for (auto& b : jb) b.free_device();
    if (d_scratch) cudaFree(d_scratch);
  }
};

namespace fbg {
LayoutParams interp_params(const fbg_program* p);
LayoutParams jit_params(const fbg_program* p);
void strip_prune(LutProgram& lp);
std::vector<int> order_for(const fbg_program* p, bool count_layout);
fbg_status build_interp(fbg_program* p, int which);
// the host half of an interpreter build (layout, LUTs, bytecode, live units)
// into the build cache, so that a later build_interp only uploads
fbg_status prebuild_interp_host(fbg_program* p, int which);
fbg_status build_jit(fbg_program* p, int mode);
fbg_status pick_engine(fbg_program* p, int mode, bool* use_jit);
// one count of units [ubegin, uend) on stream st into dev_count (null: the
// program's scratch word); the engine is picked (and built) first
fbg_status launch_count(fbg_program* p, cudaStream_t st, unsigned long long* dev_count, unsigned long long* unit_counts,
                        bool* used_jit, uint64_t ubegin = 0, uint64_t uend = ~0ull,
                        unsigned long long* unit_trace = nullptr, unsigned long long* item_trace = nullptr);
}  // namespace fbg
