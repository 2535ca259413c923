// api.cpp -- the C ABI of include/fbg.h for single programs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <sstream>

#include "build_cache.hpp"
#include "emit.hpp"
#include "fbg.h"
#include "fbg_internal.hpp"
#include "jit.hpp"
#include "kernels.hpp"
#include "program.hpp"

using namespace fbg;

namespace fbg {

thread_local std::string g_last_error;

fbg_status set_error(fbg_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

fbg_status cuda_error(cudaError_t e, const char* where) {
  return set_error(e == cudaErrorMemoryAllocation ? FBG_ENOMEM : FBG_ECUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

// SM count of the current device, cached per device (up to 64 devices)
int device_sms() {
  static std::mutex mu;
  static int sms_of[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < 64;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cached && sms_of[dev] > 0) return sms_of[dev];
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  std::lock_guard<std::mutex> lock(mu);
  if (cached) sms_of[dev] = sms;
  return sms;
}

}  // namespace fbg

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
  } while (0)

namespace fbg {

// the interpreter's layout parameters, the variable order of a layout and the
// removal of prune points: one recipe for every count path
LayoutParams interp_params(const fbg_program* p) {
  LayoutParams lp;
  lp.r_max = 1;
  lp.warps_log2 = FBG_INTERP_WARPS_LOG2;
  lp.unit_bits_max = (int)p->opt_unit_bits;
  // one letter per loop level by default: a level whose partial conjunction
  // is zero for the whole warp skips the rest, so the interpreter, whose cost
  // is per executed instruction, prunes at every letter
  lp.loop_level_bits = p->opt_loop_level_bits ? (int)p->opt_loop_level_bits : 1;
  lp.max_loop_levels = FBG_INTERP_MAX_LEVELS - 2;
  return lp;
}

LayoutParams jit_params(const fbg_program* p) {
  LayoutParams lp;
  lp.r_max = (int)p->opt_regs_log2;
  lp.warps_log2 = (int)p->opt_warps_log2;
  lp.unit_bits_max = (int)p->opt_unit_bits;
  lp.loop_level_bits = p->opt_loop_level_bits ? (int)p->opt_loop_level_bits : 4;
  lp.inner_bits = (int)p->opt_inner_bits;
  return lp;
}

void strip_prune(LutProgram& lp) {
  for (auto& li : lp.levels) li.has_acc = false;
}

std::vector<int> order_for(const fbg_program* p, bool count_layout) {
  if (count_layout && p->opt_search) return search_order(*p->g, (uint64_t)p->opt_order_seed);
  return identity_order(p->n);
}

}  // namespace fbg

namespace {

fbg_status ensure_scratch(fbg_program* p, size_t words) {
  if (p->d_scratch && p->scratch_words >= words) return FBG_OK;
  if (p->d_scratch) cudaFree(p->d_scratch);
  p->d_scratch = nullptr;
  p->scratch_words = 0;
  p->scratch_clean = false;
  CK(cudaMalloc(&p->d_scratch, words * sizeof(unsigned long long)));
  p->scratch_words = words;
  return FBG_OK;
}

}  // namespace

namespace fbg {

// the host half of an interpreter build: layout, LUTs, bytecode, item
// grouping and the units that can hold models
static std::shared_ptr<const InterpHost> interp_host(fbg_program* p, int which) {
  const std::string key = build_key(p, "interp", which);
  if (auto hit = interp_host_get(key)) return hit;
  auto h = std::make_shared<InterpHost>();
  Layout L = make_layout(p->n, interp_params(p), order_for(p, which == 0));
  h->lp = lower_and_map(*p->g, L);
  if (!p->opt_prune) strip_prune(h->lp);
  h->code = emit_bytecode(h->lp);
  const uint64_t nunits = h->code.prog.nunits;
  // work items: single units while that keeps the queue short, else ranges
  uint64_t per = 1;
  while (nunits / per > 65536) per <<= 1;
  if (p->opt_prune && nunits <= (1ull << 21)) {
    // units on which a conjunct over unit and warp letters is false have no
    // models: counts, tables (zeroed before the launch) and model lists leave
    // them out when that removes a quarter of them; the live units are then
    // single-unit items when at most 2^18 remain
    const std::vector<uint64_t> alive = alive_words(*p->g, h->lp.layout);
    const int wb = h->lp.layout.warp_bits;
    std::vector<uint32_t> live;
    if (!alive.empty()) {
      // item t = (unit << wb) | warp slice: a unit lives when any slice does
      const uint64_t nbits = nunits << wb;
      for (uint64_t t0 = 0; t0 < nbits; t0 += 64) {
        uint64_t word = alive[(size_t)(t0 >> 6)];
        if (nbits - t0 < 64) word &= (1ull << (nbits - t0)) - 1ull;
        while (word) {
          const uint64_t t = t0 + (uint64_t)__builtin_ctzll(word);
          const uint64_t u = t >> wb;
          if (live.empty() || live.back() != (uint32_t)u) live.push_back((uint32_t)u);
          word &= word - 1;
        }
      }
    }
    if (!alive.empty() && live.size() * 4 <= nunits * 3 && (per == 1 || live.size() <= (1u << 18))) {
      h->live = std::make_shared<const std::vector<uint32_t>>(std::move(live));
      per = 1;
    }
  }
  h->units_per_item = per;
  std::shared_ptr<const InterpHost> hc = std::move(h);
  interp_host_put(key, hc);
  return hc;
}

fbg_status prebuild_interp_host(fbg_program* p, int which) {
  try {
    interp_host(p, which);
  } catch (CompileError& e) {
    return set_error(FBG_ETOOBIG, e.msg);
  }
  return FBG_OK;
}

fbg_status build_interp(fbg_program* p, int which) {
  InterpBuild& b = p->ib[which];
  if (b.valid) return FBG_OK;
  std::shared_ptr<const InterpHost> h;
  try {
    h = interp_host(p, which);
  } catch (CompileError& e) {
    return set_error(FBG_ETOOBIG, e.msg);
  }
  b.lp = h->lp;
  b.code = h->code;
  b.nunits = b.code.prog.nunits;
  b.live = h->live;
  const uint64_t per = h->units_per_item;
  // the program's own item list (full-range launches); a build for the
  // server (pooled) has none: the server makes the items of every tick
  std::vector<FbgWorkItem> items;
  if (!p->alloc_stream) {
    if (per == 1)
      b.append_items(items, 0u, 0, b.live_units(), 1);
    else
      for (uint64_t u = 0; u < b.nunits; u += per) items.push_back(FbgWorkItem{0u, 0u, u, std::min(b.nunits, u + per)});
  }
  b.units_per_item = per;
  b.nitems = items.size();
  b.free_device();
  // one allocation and one copy: [descriptor][bytecode][constants][items],
  // each part 16-byte aligned
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t off_ins = al(sizeof(FbgInterpProg));
  const size_t off_consts = al(off_ins + std::max<size_t>(1, b.code.ins.size()) * 8);
  const size_t off_items = al(off_consts + std::max<size_t>(1, b.code.consts.size()) * 8);
  const size_t total = off_items + std::max<size_t>(1, items.size()) * sizeof(FbgWorkItem);
  char* base = nullptr;
  if (p->alloc_stream) {
    CK(cudaMallocAsync((void**)&base, total, p->alloc_stream));
    b.pooled = true;
    b.free_stream = p->free_stream ? p->free_stream : p->alloc_stream;
  } else {
    CK(cudaMalloc(&base, total));
  }
  b.d_prog = reinterpret_cast<FbgInterpProg*>(base);
  b.d_ins = reinterpret_cast<unsigned long long*>(base + off_ins);
  b.d_consts = reinterpret_cast<unsigned long long*>(base + off_consts);
  b.d_items = reinterpret_cast<FbgWorkItem*>(base + off_items);
  std::vector<char> staging(total, 0);
  FbgInterpProg G = b.code.prog;
  G.ins = b.d_ins;
  G.consts = b.d_consts;
  std::memcpy(staging.data(), &G, sizeof G);
  if (!b.code.ins.empty()) std::memcpy(staging.data() + off_ins, b.code.ins.data(), b.code.ins.size() * 8);
  if (!b.code.consts.empty())
    std::memcpy(staging.data() + off_consts, b.code.consts.data(), b.code.consts.size() * 8);
  if (!items.empty()) std::memcpy(staging.data() + off_items, items.data(), items.size() * sizeof(FbgWorkItem));
  if (p->alloc_stream)   // returns once the pageable source is staged
    CK(cudaMemcpyAsync(base, staging.data(), total, cudaMemcpyHostToDevice, p->alloc_stream));
  else
    CK(cudaMemcpy(base, staging.data(), total, cudaMemcpyHostToDevice));
  int per_sm = interp_blocks_per_sm(which == 0 ? 0 : 2, b.code.nslots);
  if (per_sm <= 0) return set_error(FBG_ETOOBIG, "interpreter program does not fit in shared memory");
  b.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(b.nitems, (uint64_t)device_sms() * (uint64_t)per_sm));
  b.valid = true;
  return FBG_OK;
}

// the items a full-range count hands out, uploaded in the given order
fbg_status upload_items(JitBuild& b, const std::vector<unsigned>& items) {
  b.free_device();
  CK(cudaMalloc(&b.d_perm, std::max<size_t>(1, items.size()) * sizeof(unsigned)));
  if (!items.empty())
    CK(cudaMemcpy(b.d_perm, items.data(), items.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  b.nperm = items.size();
  return FBG_OK;
}

fbg_status build_jit_impl(fbg_program* p, int mode);

fbg_status build_jit(fbg_program* p, int mode) {
  if (p->jb[mode].valid) return FBG_OK;
  const auto t0 = std::chrono::steady_clock::now();
  fbg_status s = build_jit_impl(p, mode);
  p->t_build += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

// the host half of a specialised-kernel build: layout, LUTs, source and the
// (unit, warp slice) items that can hold models
static std::shared_ptr<const JitHost> jit_host(fbg_program* p, int mode) {
  const std::string key = build_key(p, "jit", mode);
  if (auto hit = jit_host_get(key)) return hit;
  auto h = std::make_shared<JitHost>();
  const std::vector<int> ord = mode == 2 ? enum_order(p->n, jit_params(p)) : order_for(p, mode == 0);
  Layout L = make_layout(p->n, jit_params(p), ord);
  h->lp = lower_and_map(*p->g, L);
  if (!p->opt_prune) strip_prune(h->lp);
  h->block = h->lp.layout.lane_bits < 5 ? 32 : 32 << h->lp.layout.warp_bits;
  h->src = emit_cuda_source(h->lp, mode, h->block, (int)p->opt_min_blocks, &h->ops, &h->unrolled_level,
                            p->opt_stats != 0, &h->uops, (int)p->opt_popc_cost);
  if (mode == 0 && p->opt_prune) {
    // items on which a conjunct over unit and warp letters is false have no
    // models: full-range counts skip them when that removes at least a
    // quarter of the items
    h->alive = alive_items(*p->g, h->lp.layout);
    uint64_t live = 0;
    for (uint8_t a : h->alive) live += a;
    if (h->alive.empty() || live * 4 > h->alive.size() * 3) h->alive.clear();
    for (size_t t = 0; t < h->alive.size(); t++)
      if (h->alive[t]) h->items.push_back((unsigned)t);
  }
  std::shared_ptr<const JitHost> hc = std::move(h);
  jit_host_put(key, hc);
  return hc;
}

fbg_status build_jit_impl(fbg_program* p, int mode) {
  JitBuild& b = p->jb[mode];
  std::shared_ptr<const JitHost> h;
  try {
    h = jit_host(p, mode);
  } catch (CompileError& e) {
    return set_error(FBG_ETOOBIG, e.msg);
  }
  b.lp = h->lp;
  b.src = h->src;
  b.ops = h->ops;
  b.uops = h->uops;
  b.unrolled_level = h->unrolled_level;
  b.block = h->block;
  int dev = 0;
  cudaGetDevice(&dev);
  // the kernel and the live-item list of this build on this device, shared
  // with earlier programs built from the same text and options
  const std::string key = build_key(p, "jit", mode);
  std::shared_ptr<JitDevice> jd = jit_device_get(key, dev);
  if (jd) {
    b.kern = (cudaKernel_t)jd->kernel;
  } else {
    JitResult r = jit_compile(b.src, mode == 0 ? "fbg_jit_count" : mode == 1 ? "fbg_jit_table" : "fbg_jit_enum", dev);
    b.log = r.log;
    p->jit_log = r.log;
    if (!r.ok) return set_error(FBG_EJIT, r.log);
    b.kern = r.kernel;
  }
  int per_sm = jd ? jd->blocks_per_sm : 0;
  if (per_sm <= 0) {
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)b.kern, b.block, 0));
    if (per_sm <= 0) per_sm = 1;
  }
  b.nunits = 1ull << b.lp.layout.unit_bits;
  b.grid = (int)std::min<uint64_t>(b.nunits, (uint64_t)device_sms() * (uint64_t)per_sm);
  b.alive = h->alive;
  if (!h->items.empty()) {
    if (!jd || !jd->items) {
      auto nd = std::make_shared<JitDevice>();
      nd->kernel = (void*)b.kern;
      nd->blocks_per_sm = per_sm;
      unsigned* d = nullptr;
      CK(cudaMalloc(&d, h->items.size() * sizeof(unsigned)));
      nd->items = std::shared_ptr<void>(d, [](void* q) { cudaFree(q); });
      CK(cudaMemcpy(d, h->items.data(), h->items.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
      jit_device_put(key, dev, nd);
      jd = nd;
    }
    b.free_device();
    b.perm_owner = jd->items;
    b.d_perm = static_cast<unsigned*>(jd->items.get());
    b.nperm = h->items.size();
  } else if (!jd) {
    auto nd = std::make_shared<JitDevice>();
    nd->kernel = (void*)b.kern;
    nd->blocks_per_sm = per_sm;
    jit_device_put(key, dev, nd);
  }
  b.valid = true;
  return FBG_OK;
}

// which engine runs counts/tables: JIT unless the interpreter is requested
// (or, with the automatic choice, the JIT build failed)
fbg_status pick_engine(fbg_program* p, int mode, bool* use_jit) {
  if (p->opt_engine == FBG_ENGINE_INTERP) {
    *use_jit = false;
    return build_interp(p, mode == 0 ? 0 : 1);
  }
  fbg_status s = build_jit(p, mode);
  if (s == FBG_OK) {
    *use_jit = true;
    return FBG_OK;
  }
  if (p->opt_engine == FBG_ENGINE_JIT) return s;
  *use_jit = false;
  return build_interp(p, mode == 0 ? 0 : 1);
}

// scratch head: [0] item counter, [1] count of fbg_count, [2] [3] interpreter
// item counter and total, [4..20) level iterations, [24] [25] running sum and
// finished warps of self-resetting counts; then, for model lists and
// interpreter sub-ranges, arrays after the head
constexpr size_t kScratchHead = 32;
constexpr size_t kScratchAcc = 24, kScratchDone = 25;

fbg_status launch_count(fbg_program* p, cudaStream_t st, unsigned long long* dev_count, unsigned long long* unit_counts,
                        bool* used_jit, uint64_t ubegin, uint64_t uend, unsigned long long* unit_trace,
                        unsigned long long* item_trace) {
  bool jit = false;
  fbg_status s = pick_engine(p, 0, &jit);
  if (s != FBG_OK) return s;
  if (p->n > 63) return set_error(FBG_ETOOBIG, "counts need n <= 63");
  size_t words = kScratchHead;
  if (!jit) {   // room for the work items of a sub-range (interpreter)
    const InterpBuild& ib = p->ib[0];
    uint64_t e = std::min<uint64_t>(uend, ib.nunits);
    if (e > ubegin && !(ubegin == 0 && e == ib.nunits))
      words += ((e - ubegin) / ib.units_per_item + 2) * (sizeof(FbgWorkItem) / 8) + 1;
  }
  s = ensure_scratch(p, words);
  if (s != FBG_OK) return s;
  if (!dev_count) dev_count = p->d_scratch + 1;
  if (p->g->root == 0 || p->g->root == 1) {
    // the Reduction left a constant: every assignment of a unit is a model
    // (true) or none is (false), so the counts are written without an
    // evaluation (2^n models for a tautology, up to 2^63)
    const Layout& L = jit ? p->jb[0].lp.layout : p->ib[0].lp.layout;
    const uint64_t nunits = 1ull << L.unit_bits;
    const uint64_t e = std::min<uint64_t>(uend, nunits);
    if (ubegin > e) return set_error(FBG_EINVAL, "empty or inverted unit range");
    const uint64_t per_unit = p->g->root == 1 ? (1ull << (p->n - L.unit_bits)) : 0ull;
    CK(cudaMemsetAsync(p->d_scratch, 0, kScratchHead * 8, st));
    p->scratch_clean = true;
    CK(launch_fill_u64(dev_count, 1, (e - ubegin) * per_unit, st));
    if (unit_counts) CK(launch_fill_u64(unit_counts, e - ubegin, per_unit, st));
    *used_jit = jit;
    return FBG_OK;
  }
  // a plain count of a non-empty range with the NVRTC engine resets its own
  // counters and writes the total: no memset is needed once the head is clean
  bool self_reset = false;
  if (jit) {
    const uint64_t e = std::min<uint64_t>(uend, p->jb[0].nunits);
    self_reset = !unit_counts && !unit_trace && !item_trace && !p->opt_stats && e > ubegin;
  }
  if (!self_reset || !p->scratch_clean) CK(cudaMemsetAsync(p->d_scratch, 0, kScratchHead * 8, st));
  if (!self_reset && dev_count != p->d_scratch + 1) CK(cudaMemsetAsync(dev_count, 0, 8, st));
  p->scratch_clean = false;
  FbgLaunch P{};
  P.count = self_reset ? nullptr : dev_count;
  P.unit_counts = unit_counts;
  P.unit_ctr = p->d_scratch + 0;
  P.iters = p->opt_stats ? p->d_scratch + 4 : nullptr;
  P.unit_begin = 0;
  if (jit) {
    JitBuild& b = p->jb[0];
    uend = std::min<uint64_t>(uend, b.nunits);
    if (ubegin > uend) return set_error(FBG_EINVAL, "empty or inverted unit range");
    P.unit_begin = ubegin;
    P.unit_end = uend;
    P.unit_trace = unit_trace;
    P.item_trace = item_trace;
    // a few fetches per resident block and unit: enough to balance pruned work
    P.chunk = std::max<uint64_t>(1, (uend - ubegin) / ((uint64_t)b.grid * 16));
    // the item list (live units, measured order) covers full-range counts
    // without per-unit outputs; a list shorter than the grid's warps gets
    // only the blocks it needs (every warp of a launch draws from the item
    // counter and reports to the finish counter once)
    uint64_t grid = (uint64_t)b.grid;
    if (b.d_perm && ubegin == 0 && uend == b.nunits && !unit_counts && !unit_trace && !item_trace) {
      P.unit_perm = b.d_perm;
      P.nperm = b.nperm;
      const uint64_t wpb = (uint64_t)(b.block / 32);
      grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (b.nperm + wpb - 1) / wpb));
      P.chunk = std::max<uint64_t>(1, b.nperm / (grid * wpb * 16));
    }
    if (self_reset) {
      P.acc = p->d_scratch + kScratchAcc;
      P.done = p->d_scratch + kScratchDone;
      P.out = dev_count;
      P.nwarps = (fbg_u32)(grid * (uint64_t)b.block / 32);
    }
    void* args[] = {&P};
    if (uend > ubegin)
      CK(cudaLaunchKernel((const void*)b.kern, dim3((unsigned)grid), dim3((unsigned)b.block), args, 0, st));
    p->scratch_clean = self_reset;
  } else {
    InterpBuild& b = p->ib[0];
    uend = std::min<uint64_t>(uend, b.nunits);
    if (ubegin > uend) return set_error(FBG_EINVAL, "empty or inverted unit range");
    if (unit_counts && b.units_per_item != 1) return set_error(FBG_ETOOBIG, "too many units for per-unit counts");
    P.unit_end = b.nunits;
    if (ubegin == 0 && uend == b.nunits) {
      CK(launch_interp(0, b.d_prog, b.d_items, b.nitems, p->d_scratch + 2, dev_count, unit_counts, P, b.code.nslots,
                       b.grid, st));
    } else if (uend > ubegin) {
      // a sub-range: items aligned to the program's item grouping, clipped at the ends
      std::vector<FbgWorkItem> items;
      for (uint64_t u = ubegin; u < uend;) {
        uint64_t e = std::min(uend, (u / b.units_per_item + 1) * b.units_per_item);
        items.push_back(FbgWorkItem{0u, 0u, u, e});
        u = e;
      }
      FbgWorkItem* d_items = reinterpret_cast<FbgWorkItem*>(p->d_scratch + kScratchHead);
      CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(FbgWorkItem), cudaMemcpyHostToDevice, st));
      int grid = (int)std::min<uint64_t>(items.size(), (uint64_t)b.grid);
      CK(launch_interp(0, b.d_prog, d_items, items.size(), p->d_scratch + 2, dev_count, unit_counts, P, b.code.nslots,
                       grid, st));
      CK(cudaStreamSynchronize(st));   // the host item list goes out of scope
    }
  }
  *used_jit = jit;
  return FBG_OK;
}

}  // namespace fbg

// executed work of the last launch from its level counters (scratch head
// words 4..19, FBG_OPT_STATS = 1): per level, executions x the lop3.b32 the
// kernel issues per execution (JIT: the folded source's lane-varying ops;
// interpreter: two per instruction for its 64-bit tiles)
static void fill_exec_stats(fbg_program* p, bool jit, int mode, const unsigned long long* host) {
  fbg_exec_stats& es = p->last;
  std::memset(&es, 0, sizeof es);
  es.engine = jit ? FBG_ENGINE_JIT : FBG_ENGINE_INTERP;
  if (!p->opt_stats) return;
  const JitBuild& jb = p->jb[mode];
  const LutProgram& lp = jit ? jb.lp : p->ib[mode].lp;
  const Layout& L = lp.layout;
  double execs = (double)(1ull << L.unit_bits) * (double)(1 << L.warp_bits);
  for (int lv = 0; lv < L.nlevels() && lv < 16; lv++) {
    es.level_iters[lv] = host[4 + lv];
    double per = jit ? (double)jb.ops[(size_t)lv] * 32.0
                     : (double)(lp.levels[(size_t)lv].lut_end - lp.levels[(size_t)lv].lut_begin) * 64.0;
    es.lop3_executed += (double)host[4 + lv] * per;
    if (jit) es.lop3_uniform += (double)host[4 + lv] * (double)jb.uops[(size_t)lv];
    if (lv >= 2 && !(jit && lv == jb.unrolled_level)) execs *= (double)(1u << L.loop_bits[(size_t)(lv - 2)]);
    double nominal_execs = lv == 0 ? 0.0 : execs;
    es.lop3_nominal += nominal_execs * (jit ? (double)(jb.ops[(size_t)lv] + jb.uops[(size_t)lv]) * 32.0 : per);
  }
}

// ------------------------------------------------------------------ ABI --

extern "C" {

fbg_status fbg_compile(const char* formula, int domain_k, fbg_program** out) {
  if (!formula || !out) return set_error(FBG_EINVAL, "null argument");
  *out = nullptr;
  auto* p = new fbg_program();
  try {
    p->compiled = compile_cached(formula, domain_k);
    p->th = &p->compiled->th;
    p->g = &p->compiled->g;
  } catch (CompileError& e) {
    delete p;
    bool big = e.msg.find("more than") != std::string::npos;
    return set_error(big ? FBG_ETOOBIG : FBG_EPARSE, e.msg);
  }
  p->text = formula;
  p->k = domain_k;
  p->n = p->g->nvars;
  *out = p;
  return FBG_OK;
}

int fbg_num_vars(const fbg_program* p) { return p ? p->n : -1; }

fbg_status fbg_var_name(const fbg_program* p, int i, char* buf, size_t len) {
  if (!p || !buf || i < 0 || i >= p->n) return set_error(FBG_EINVAL, "bad variable index");
  const std::string& s = p->th->var_names[(size_t)p->g->letter_of_var[(size_t)i]];
  if (len < s.size() + 1) return set_error(FBG_EINVAL, "buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return FBG_OK;
}

fbg_status fbg_set_option(fbg_program* p, int option, int64_t v) {
  if (!p) return set_error(FBG_EINVAL, "null program");
  auto bad = [] { return set_error(FBG_EINVAL, "option value out of range"); };
  switch (option) {
    case FBG_OPT_ENGINE:
      if (v < 0 || v > 2) return bad();
      p->opt_engine = v;
      break;
    case FBG_OPT_PRUNE: p->opt_prune = v ? 1 : 0; break;
    case FBG_OPT_REGS_LOG2:
      if (v < 1 || v > 3) return bad();
      p->opt_regs_log2 = v;
      break;
    case FBG_OPT_WARPS_LOG2:
      if (v < 0 || v > 5) return bad();
      p->opt_warps_log2 = v;
      break;
    case FBG_OPT_UNIT_BITS:
      if (v < 0 || v > 24) return bad();
      p->opt_unit_bits = v;
      break;
    case FBG_OPT_LOOP_LEVEL_BITS:
      if (v < 0 || v > 16) return bad();
      p->opt_loop_level_bits = v;
      break;
    case FBG_OPT_SEARCH_ORDER: p->opt_search = v ? 1 : 0; break;
    case FBG_OPT_MIN_BLOCKS:
      if (v < 1 || v > 32) return bad();
      p->opt_min_blocks = v;
      break;
    case FBG_OPT_INNER_BITS:
      if (v < 0 || v > 5) return bad();
      p->opt_inner_bits = v;
      break;
    case FBG_OPT_POPC_COST:
      if (v < 0 || v > 16) return bad();
      p->opt_popc_cost = v;
      break;
    case FBG_OPT_ORDER_SEED:
      if (v < 0 || v > 255) return bad();
      p->opt_order_seed = v;
      break;
    case FBG_OPT_SPLIT_ITEMS:   // read by the next fbg_schedule_units; kernels stay valid
      p->opt_split_items = v ? 1 : 0;
      return FBG_OK;
    case FBG_OPT_STATS:   // kernels carry level counters only while statistics are on
      if (p->opt_stats == (v ? 1 : 0)) return FBG_OK;
      p->opt_stats = v ? 1 : 0;
      break;
    default: return set_error(FBG_EINVAL, "unknown option");
  }
  p->invalidate();
  return FBG_OK;
}

fbg_status fbg_program_stats(fbg_program* p, fbg_stats* out) {
  if (!p || !out) return set_error(FBG_EINVAL, "null argument");
  std::memset(out, 0, sizeof *out);
  out->n = p->n;
  out->domain_k = p->k;
  out->dag_nodes = p->g->dag.size();
  LutProgram lp;
  try {
    Layout L = make_layout(p->n, jit_params(p), order_for(p, true));
    lp = lower_and_map(*p->g, L);
    if (!p->opt_prune) strip_prune(lp);   // as the count kernel is built
  } catch (CompileError& e) {
    return set_error(FBG_ETOOBIG, e.msg);
  }
  out->gates = lp.gates;
  out->luts = (int64_t)lp.luts.size();
  out->nlevels = lp.layout.nlevels();
  std::vector<long long> ops;
  emit_cuda_source(lp, 0, 32 << lp.layout.warp_bits, (int)p->opt_min_blocks, &ops);
  for (int i = 0; i < 16 && i < out->nlevels; i++) out->lop3_per_level[i] = ops[(size_t)i];
  out->regs_log2 = lp.layout.r;
  out->lane_bits = lp.layout.lane_bits;
  out->warp_bits = lp.layout.warp_bits;
  out->unit_bits = lp.layout.unit_bits;
  for (size_t i = 0; i < lp.layout.loop_bits.size() && i < 8; i++) out->loop_bits[i] = lp.layout.loop_bits[i];
  if (build_interp(p, 0) == FBG_OK) out->interp_slots = (int)p->ib[0].code.nslots;
  return FBG_OK;
}

fbg_status fbg_count(fbg_program* p, void* stream, uint64_t* out_count) {
  if (!p || !out_count) return set_error(FBG_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  bool jit = false;
  const auto t0 = std::chrono::steady_clock::now();
  const double build0 = p->t_build;
  fbg_status s = launch_count(p, st, nullptr, nullptr, &jit);
  if (s != FBG_OK) return s;
  unsigned long long host[kScratchHead];
  CK(cudaMemcpyAsync(host, p->d_scratch, sizeof host, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  p->t_count += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() - (p->t_build - build0);
  *out_count = host[1];
  fill_exec_stats(p, jit, 0, host);
  return FBG_OK;
}

fbg_status fbg_count_range(fbg_program* p, void* stream, uint64_t unit_begin, uint64_t unit_end, uint64_t* out_count) {
  if (!p || !out_count) return set_error(FBG_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  bool jit = false;
  fbg_status s = launch_count(p, st, nullptr, nullptr, &jit, unit_begin, unit_end);
  if (s != FBG_OK) return s;
  unsigned long long c = 0;
  CK(cudaMemcpyAsync(&c, p->d_scratch + 1, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *out_count = c;
  return FBG_OK;
}

fbg_status fbg_count_async(fbg_program* p, void* stream, uint64_t* dev_out) {
  if (!p || !dev_out) return set_error(FBG_EINVAL, "null argument");
  bool jit = false;
  return launch_count(p, (cudaStream_t)stream, (unsigned long long*)dev_out, nullptr, &jit);
}

fbg_status fbg_count_each(fbg_program** progs, size_t nprogs, void* stream, uint64_t* dev_out) {
  if ((!progs || !dev_out) && nprogs) return set_error(FBG_EINVAL, "null argument");
  for (size_t i = 0; i < nprogs; i++) {
    if (!progs[i]) return set_error(FBG_EINVAL, "null program");
    bool jit = false;
    fbg_status s = launch_count(progs[i], (cudaStream_t)stream, (unsigned long long*)(dev_out + i), nullptr, &jit);
    if (s != FBG_OK) return s;
  }
  return FBG_OK;
}

fbg_status fbg_unit_vars(fbg_program* p, int* vars, int max_vars, int* nvars, uint64_t* nunits) {
  if (!p || !nvars || !nunits) return set_error(FBG_EINVAL, "null argument");
  bool jit = false;
  fbg_status s = pick_engine(p, 0, &jit);
  if (s != FBG_OK) return s;
  const Layout& L = jit ? p->jb[0].lp.layout : p->ib[0].lp.layout;
  *nvars = L.unit_bits;
  *nunits = 1ull << L.unit_bits;
  for (int b = 0; b < L.unit_bits && b < max_vars; b++) vars[b] = L.var_of_pos[(size_t)(L.first_unit_pos() + b)];
  return FBG_OK;
}

fbg_status fbg_count_units(fbg_program* p, void* stream, uint64_t* dev_counts, uint64_t nunits) {
  if (!p || !dev_counts) return set_error(FBG_EINVAL, "null argument");
  int vars[64], nv = 0;
  uint64_t nu = 0;
  fbg_status s = fbg_unit_vars(p, vars, 64, &nv, &nu);
  if (s != FBG_OK) return s;
  if (nunits != nu) return set_error(FBG_EINVAL, "nunits must be " + std::to_string(nu));
  cudaStream_t st = (cudaStream_t)stream;
  s = ensure_scratch(p, kScratchHead);
  if (s != FBG_OK) return s;
  CK(cudaMemsetAsync(dev_counts, 0, nunits * 8, st));
  bool jit = false;
  s = launch_count(p, st, nullptr, (unsigned long long*)dev_counts, &jit);
  if (s != FBG_OK) return s;
  CK(cudaStreamSynchronize(st));
  return FBG_OK;
}

fbg_status fbg_schedule_units(fbg_program* p, void* stream) {
  if (!p) return set_error(FBG_EINVAL, "null argument");
  if (p->n > 63) return set_error(FBG_ETOOBIG, "counts need n <= 63");
  bool jit = false;
  fbg_status s = pick_engine(p, 0, &jit);
  if (s != FBG_OK) return s;
  if (!jit) return set_error(FBG_EINVAL, "unit schedules need the NVRTC engine");
  JitBuild& b = p->jb[0];
  const int wb = b.lp.layout.warp_bits;
  const uint64_t items = b.nunits << wb;
  if (items > (1ull << 24)) return set_error(FBG_ETOOBIG, "too many items to schedule");
  cudaStream_t st = (cudaStream_t)stream;
  s = ensure_scratch(p, kScratchHead);
  if (s != FBG_OK) return s;
  b.free_device();   // measure in the natural order
  unsigned long long* d_tr = nullptr;
  CK(cudaMalloc(&d_tr, items * 8));
  std::vector<uint64_t> ns((size_t)items);
  cudaError_t e = cudaMemsetAsync(d_tr, 0, items * 8, st);
  if (e == cudaSuccess) {
    s = launch_count(p, st, nullptr, nullptr, &jit, 0, ~0ull, nullptr, d_tr);
    if (s == FBG_OK) e = cudaMemcpyAsync(ns.data(), d_tr, items * 8, cudaMemcpyDeviceToHost, st);
    if (s == FBG_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(d_tr);
  if (s != FBG_OK) return s;
  if (e != cudaSuccess) return cuda_error(e, "fbg_schedule_units trace");
  // units without models (b.alive) stay out
  std::vector<unsigned> live;
  live.reserve((size_t)items);
  double sum = 0;
  for (uint64_t t = 0; t < items; t++)
    if (b.alive.empty() || b.alive[(size_t)t]) {
      live.push_back((unsigned)t);
      sum += (double)ns[(size_t)t];
    }
  // An item longer than half the mean load of a warp would end the launch
  // late on its own: it is handed out as 2^s pieces over the first loop level
  // (each estimated at its share of the item's time).
  const int smax = p->opt_split_items ? top_loop_split_bits(b.lp.layout) : 0;
  const double warps = (double)b.grid * (double)(b.block / 32);
  const double target = sum / warps / 2.0;
  struct Piece {
    unsigned code;
    double t;
  };
  std::vector<Piece> pieces;
  pieces.reserve(live.size());
  for (unsigned t : live) {
    const double d = (double)ns[t];
    int sb = 0;
    while (sb < smax && d / (double)(1u << sb) > target) sb++;
    for (unsigned q = 0; q < (1u << sb); q++)
      pieces.push_back(Piece{t | ((unsigned)sb << 28) | (q << 24), d / (double)(1u << sb)});
  }
  // longest processing time first; ties keep the natural (unit, slice, piece) order
  std::stable_sort(pieces.begin(), pieces.end(), [](const Piece& x, const Piece& y) { return x.t > y.t; });
  std::vector<unsigned> perm(pieces.size());
  for (size_t i = 0; i < pieces.size(); i++) perm[i] = pieces[i].code;
  return upload_items(b, perm);
}

fbg_status fbg_debug_host_caches(int clear, uint64_t out[9]) {
  if (!out) return set_error(FBG_EINVAL, "null argument");
  if (clear) host_caches_clear();
  host_cache_stats(out);
  return FBG_OK;
}

fbg_status fbg_debug_host_times(const fbg_program* p, double* build_s, double* count_s) {
  if (!p || !build_s || !count_s) return set_error(FBG_EINVAL, "null argument");
  *build_s = p->t_build;
  *count_s = p->t_count;
  return FBG_OK;
}

fbg_status fbg_debug_item_trace(fbg_program* p, void* stream, uint64_t* dev_ns, uint64_t nitems) {
  if (!p || !dev_ns) return set_error(FBG_EINVAL, "null argument");
  bool jit = false;
  fbg_status s = pick_engine(p, 0, &jit);
  if (s != FBG_OK) return s;
  if (!jit) return set_error(FBG_EINVAL, "item traces need the NVRTC engine");
  const JitBuild& b = p->jb[0];
  const uint64_t items = b.nunits << b.lp.layout.warp_bits;
  if (nitems != items) return set_error(FBG_EINVAL, "nitems must be " + std::to_string(items));
  cudaStream_t st = (cudaStream_t)stream;
  s = ensure_scratch(p, kScratchHead);
  if (s != FBG_OK) return s;
  CK(cudaMemsetAsync(dev_ns, 0, items * 8, st));
  s = launch_count(p, st, nullptr, nullptr, &jit, 0, ~0ull, nullptr, (unsigned long long*)dev_ns);
  if (s != FBG_OK) return s;
  CK(cudaStreamSynchronize(st));
  return FBG_OK;
}

fbg_status fbg_debug_unit_trace(fbg_program* p, void* stream, uint64_t* dev_trace, uint64_t nunits) {
  if (!p || !dev_trace) return set_error(FBG_EINVAL, "null argument");
  int vars[64], nv = 0;
  uint64_t nu = 0;
  fbg_status s = fbg_unit_vars(p, vars, 64, &nv, &nu);
  if (s != FBG_OK) return s;
  if (nunits != nu) return set_error(FBG_EINVAL, "nunits must be " + std::to_string(nu));
  bool jit = false;
  s = pick_engine(p, 0, &jit);
  if (s != FBG_OK) return s;
  if (!jit) return set_error(FBG_EINVAL, "unit traces need the NVRTC engine");
  cudaStream_t st = (cudaStream_t)stream;
  // durations 0, start times all-ones (the kernel takes the minimum)
  CK(cudaMemsetAsync(dev_trace, 0xFF, nunits * 16, st));
  CK(cudaMemset2DAsync(dev_trace, 16, 0, 8, nunits, st));
  s = launch_count(p, st, nullptr, nullptr, &jit, 0, ~0ull, (unsigned long long*)dev_trace);
  if (s != FBG_OK) return s;
  CK(cudaStreamSynchronize(st));
  return FBG_OK;
}

fbg_status fbg_truth_table(fbg_program* p, void* stream, uint64_t* dev_words, size_t nwords) {
  if (!p || !dev_words) return set_error(FBG_EINVAL, "null argument");
  if (p->n > 40) return set_error(FBG_ETOOBIG, "truth tables need n <= 40");
  size_t need = p->n <= 6 ? 1 : (size_t)1 << (p->n - 6);
  if (nwords != need) return set_error(FBG_EINVAL, "nwords must be " + std::to_string(need));
  cudaStream_t st = (cudaStream_t)stream;
  bool jit = false;
  fbg_status s = pick_engine(p, 1, &jit);
  if (s != FBG_OK) return s;
  s = ensure_scratch(p, kScratchHead);
  if (s != FBG_OK) return s;
  CK(cudaMemsetAsync(p->d_scratch, 0, kScratchHead * 8, st));
  p->scratch_clean = false;
  FbgLaunch P{};
  P.table = (fbg_u32*)dev_words;
  P.unit_ctr = p->d_scratch + 0;
  P.unit_begin = 0;
  if (jit) {
    JitBuild& b = p->jb[1];
    if (p->n < 6) CK(cudaMemsetAsync(dev_words, 0, 8, st));
    P.unit_end = b.nunits;
    P.chunk = std::max<uint64_t>(1, b.nunits / ((uint64_t)b.grid * 16));
    P.iters = p->opt_stats ? p->d_scratch + 4 : nullptr;
    void* args[] = {&P};
    CK(cudaLaunchKernel((const void*)b.kern, dim3((unsigned)b.grid), dim3((unsigned)b.block), args, 0, st));
    if (p->opt_stats) {   // executed work of this table (fbg_last_exec_stats)
      unsigned long long host[kScratchHead];
      CK(cudaMemcpyAsync(host, p->d_scratch, sizeof host, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      fill_exec_stats(p, true, 1, host);
    }
  } else {
    InterpBuild& b = p->ib[1];
    CK(cudaMemsetAsync(dev_words, 0, nwords * 8, st));
    P.unit_end = b.nunits;
    CK(launch_interp(1, b.d_prog, b.d_items, b.nitems, p->d_scratch + 2, nullptr, nullptr, P, b.code.nslots, b.grid,
                     st));
  }
  return FBG_OK;
}

// Model list with the specialised kernel (layout of enum_order): pass 1 counts
// the models of every (unit, warp slice) item, a scan turns the counts into
// each item's first position, pass 2 writes the models of the items that
// start below `cap`.
static fbg_status enumerate_jit(fbg_program* p, cudaStream_t st, uint64_t* dev_models, size_t cap, uint64_t* total,
                                uint64_t* written, uint64_t ubegin = 0, uint64_t uend = ~0ull) {
  JitBuild& b = p->jb[2];
  uend = std::min<uint64_t>(uend, b.nunits);
  const uint64_t nitems = (uend - ubegin) << b.lp.layout.warp_bits;
  if (nitems > (1ull << 26)) return set_error(FBG_ETOOBIG, "too many work items for a model list");
  fbg_status s = ensure_scratch(p, kScratchHead + 2 * nitems);
  if (s != FBG_OK) return s;
  unsigned long long* item_counts = p->d_scratch + kScratchHead;
  unsigned long long* offsets = item_counts + nitems;
  CK(cudaMemsetAsync(p->d_scratch, 0, kScratchHead * 8, st));
  p->scratch_clean = false;
  FbgLaunch P{};
  P.unit_ctr = p->d_scratch + 0;
  P.unit_begin = ubegin;
  P.unit_end = uend;
  P.unit_counts = item_counts;
  P.iters = p->opt_stats ? p->d_scratch + 4 : nullptr;
  const uint64_t wpb = (uint64_t)(b.block / 32);
  P.chunk = std::max<uint64_t>(1, nitems / ((uint64_t)b.grid * wpb * 16));
  void* args[] = {&P};
  CK(cudaLaunchKernel((const void*)b.kern, dim3((unsigned)b.grid), dim3((unsigned)b.block), args, 0, st));
  CK(launch_scan(item_counts, offsets, nitems, p->d_scratch + 3, st));
  if (cap) {
    CK(cudaMemsetAsync(p->d_scratch + 0, 0, 8, st));
    P.models = (unsigned long long*)dev_models;
    P.cap = cap;
    P.unit_offsets = offsets;
    CK(cudaLaunchKernel((const void*)b.kern, dim3((unsigned)b.grid), dim3((unsigned)b.block), args, 0, st));
  }
  unsigned long long tot = 0;
  CK(cudaMemcpyAsync(&tot, p->d_scratch + 3, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *total = tot;
  *written = std::min<uint64_t>(tot, cap);
  return FBG_OK;
}

fbg_status fbg_table_units(fbg_program* p, int mode, uint64_t* nunits, uint64_t* words_per_unit) {
  if (!p || !nunits || !words_per_unit || (mode != 1 && mode != 2)) return set_error(FBG_EINVAL, "bad argument");
  if (p->n > 40) return set_error(FBG_ETOOBIG, "truth tables and model lists need n <= 40");
  if (p->opt_engine == FBG_ENGINE_INTERP) return set_error(FBG_EINVAL, "unit ranges need the specialised kernel");
  fbg_status s = build_jit(p, mode);
  if (s != FBG_OK) return s;
  const Layout& L = p->jb[mode].lp.layout;
  *nunits = 1ull << L.unit_bits;
  const int below = p->n - L.unit_bits;   // letters inside one unit
  *words_per_unit = below <= 6 ? 1ull : 1ull << (below - 6);
  return FBG_OK;
}

fbg_status fbg_truth_table_range(fbg_program* p, void* stream, uint64_t unit_begin, uint64_t unit_end,
                                 uint64_t* dev_words, size_t nwords) {
  if (!p || !dev_words) return set_error(FBG_EINVAL, "null argument");
  uint64_t nunits = 0, wpu = 0;
  fbg_status s = fbg_table_units(p, 1, &nunits, &wpu);
  if (s != FBG_OK) return s;
  if (unit_begin >= unit_end || unit_end > nunits) return set_error(FBG_EINVAL, "empty or out-of-range unit range");
  if (nunits > 1 && (p->n - p->jb[1].lp.layout.unit_bits) < 6)
    return set_error(FBG_EINVAL, "units smaller than one 64-bit word: take the whole table");
  const uint64_t need = (unit_end - unit_begin) * wpu;
  if (nwords != need) return set_error(FBG_EINVAL, "nwords must be " + std::to_string(need));
  cudaStream_t st = (cudaStream_t)stream;
  s = ensure_scratch(p, kScratchHead);
  if (s != FBG_OK) return s;
  CK(cudaMemsetAsync(p->d_scratch, 0, kScratchHead * 8, st));
  p->scratch_clean = false;
  JitBuild& b = p->jb[1];
  if (p->n < 6) CK(cudaMemsetAsync(dev_words, 0, 8, st));
  FbgLaunch P{};
  P.table = (fbg_u32*)dev_words;
  P.table_word0 = unit_begin * wpu;
  P.unit_ctr = p->d_scratch + 0;
  P.unit_begin = unit_begin;
  P.unit_end = unit_end;
  const uint64_t grid = std::min<uint64_t>((uint64_t)b.grid, unit_end - unit_begin);
  P.chunk = std::max<uint64_t>(1, (unit_end - unit_begin) / (grid * 16));
  void* args[] = {&P};
  CK(cudaLaunchKernel((const void*)b.kern, dim3((unsigned)grid), dim3((unsigned)b.block), args, 0, st));
  return FBG_OK;
}

fbg_status fbg_enumerate_models_range(fbg_program* p, void* stream, uint64_t unit_begin, uint64_t unit_end,
                                      uint64_t* dev_models, size_t cap, uint64_t* total, uint64_t* written) {
  if (!p || !total || !written || (cap && !dev_models)) return set_error(FBG_EINVAL, "null argument");
  uint64_t nunits = 0, wpu = 0;
  fbg_status s = fbg_table_units(p, 2, &nunits, &wpu);
  if (s != FBG_OK) return s;
  if (unit_begin >= unit_end || unit_end > nunits) return set_error(FBG_EINVAL, "empty or out-of-range unit range");
  return enumerate_jit(p, (cudaStream_t)stream, dev_models, cap, total, written, unit_begin, unit_end);
}

fbg_status fbg_enumerate_models(fbg_program* p, void* stream, uint64_t* dev_models, size_t cap, uint64_t* total,
                                uint64_t* written) {
  if (!p || !total || !written || (cap && !dev_models)) return set_error(FBG_EINVAL, "null argument");
  if (p->n > 40) return set_error(FBG_ETOOBIG, "model lists need n <= 40");
  cudaStream_t st = (cudaStream_t)stream;
  // the specialised kernel unless the interpreter is asked for (or, with the
  // automatic choice, the specialised build fails)
  if (p->opt_engine != FBG_ENGINE_INTERP) {
    fbg_status s = build_jit(p, 2);
    if (s == FBG_OK) return enumerate_jit(p, st, dev_models, cap, total, written);
    if (p->opt_engine == FBG_ENGINE_JIT) return s;
  }
  fbg_status s = build_interp(p, 1);
  if (s != FBG_OK) return s;
  InterpBuild& b = p->ib[1];
  if (b.units_per_item != 1) return set_error(FBG_ETOOBIG, "too many units");
  s = ensure_scratch(p, kScratchHead + 2 * b.nunits);
  if (s != FBG_OK) return s;
  unsigned long long* unit_counts = p->d_scratch + kScratchHead;
  unsigned long long* offsets = unit_counts + b.nunits;
  CK(cudaMemsetAsync(p->d_scratch, 0, (kScratchHead + b.nunits) * 8, st));
  p->scratch_clean = false;
  FbgLaunch P{};
  P.unit_ctr = p->d_scratch + 0;
  P.unit_begin = 0;
  P.unit_end = b.nunits;
  // pass 1: models per unit
  CK(launch_interp(0, b.d_prog, b.d_items, b.nitems, p->d_scratch + 2, nullptr, unit_counts, P, b.code.nslots, b.grid,
                   st));
  // exclusive scan -> offsets, total
  CK(launch_scan(unit_counts, offsets, b.nunits, p->d_scratch + 3, st));
  // pass 2: ordered write
  CK(cudaMemsetAsync(p->d_scratch + 2, 0, 8, st));
  P.models = (unsigned long long*)dev_models;
  P.cap = cap;
  P.unit_offsets = offsets;
  CK(launch_interp(2, b.d_prog, b.d_items, b.nitems, p->d_scratch + 2, nullptr, nullptr, P, b.code.nslots, b.grid, st));
  unsigned long long tot = 0;
  CK(cudaMemcpyAsync(&tot, p->d_scratch + 3, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *total = tot;
  *written = std::min<uint64_t>(tot, cap);
  return FBG_OK;
}

fbg_status fbg_last_exec_stats(fbg_program* p, fbg_exec_stats* out) {
  if (!p || !out) return set_error(FBG_EINVAL, "null argument");
  *out = p->last;
  return FBG_OK;
}

fbg_status fbg_program_source(fbg_program* p, int mode, char* buf, size_t* len) {
  if (!p || !len || mode < 0 || mode > 2) return set_error(FBG_EINVAL, "bad argument");
  std::string src;
  try {
    src = jit_host(p, mode)->src;   // exactly the source the kernel build compiles
  } catch (CompileError& e) {
    return set_error(FBG_ETOOBIG, e.msg);
  }
  if (buf) {
    if (*len < src.size() + 1) return set_error(FBG_EINVAL, "buffer too small");
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  *len = src.size() + 1;
  return FBG_OK;
}

fbg_status fbg_debug_dump(fbg_program* p, int which, char* buf, size_t* len) {
  if (!p || !len || which < 0 || which > 4) return set_error(FBG_EINVAL, "bad argument");
  std::ostringstream o;
  auto layout_json = [&](const Layout& L) {
    o << "\"layout\": {\"n\": " << L.n << ", \"r\": " << L.r << ", \"lane_bits\": " << L.lane_bits
      << ", \"warp_bits\": " << L.warp_bits << ", \"unit_bits\": " << L.unit_bits
      << ", \"split_bits\": " << top_loop_split_bits(L) << ", \"loop_bits\": [";
    for (size_t i = 0; i < L.loop_bits.size(); i++) o << (i ? ", " : "") << L.loop_bits[i];
    o << "], \"loop_pos\": [";
    for (size_t i = 0; i < L.loop_bits.size(); i++) o << (i ? ", " : "") << L.loop_pos((int)i);
    o << "], \"first_unit_pos\": " << L.first_unit_pos() << ", \"pos_of_var\": [";
    for (int i = 0; i < L.n; i++) o << (i ? ", " : "") << L.pos_of_var[(size_t)i];
    o << "]}";
  };
  auto val_json = [&](const Val& v) { o << "[" << (int)v.kind << ", " << v.id << "]"; };
  if (which < 2 || which == 4) {
    LutProgram lp;
    try {
      Layout L = make_layout(p->n, jit_params(p),
                             which == 4 ? enum_order(p->n, jit_params(p)) : order_for(p, which == 0));
      lp = lower_and_map(*p->g, L);
      if (!p->opt_prune) strip_prune(lp);
    } catch (CompileError& e) {
      return set_error(FBG_ETOOBIG, e.msg);
    }
    o << "{";
    layout_json(lp.layout);
    o << ", \"consts\": [";
    for (size_t i = 0; i < lp.consts.size(); i++) {
      o << (i ? ", " : "") << "[";
      for (size_t j = 0; j < lp.consts[i].w.size(); j++) o << (j ? ", " : "") << lp.consts[i].w[j];
      o << "]";
    }
    o << "], \"luts\": [";
    for (size_t i = 0; i < lp.luts.size(); i++) {
      const Lut& lu = lp.luts[i];
      o << (i ? ", " : "") << "[" << (int)lu.tt << ", ";
      val_json(lu.in[0]);
      o << ", ";
      val_json(lu.in[1]);
      o << ", ";
      val_json(lu.in[2]);
      o << ", " << lu.level << ", " << lu.rmask << "]";
    }
    o << "], \"levels\": [";
    for (size_t i = 0; i < lp.levels.size(); i++) {
      const LevelInfo& li = lp.levels[i];
      o << (i ? ", " : "") << "[" << li.lut_begin << ", " << li.lut_end << ", " << (li.has_acc ? 1 : 0) << ", ";
      val_json(li.acc);
      o << "]";
    }
    o << "], \"out\": ";
    val_json(lp.out);
    o << ", \"const_acc\": [";
    for (size_t j = 0; j < lp.const_acc.w.size(); j++) o << (j ? ", " : "") << lp.const_acc.w[j];
    o << "]";
    if (which == 0 && p->opt_prune) {   // units the count kernel hands out (all when absent)
      std::vector<uint8_t> alive = alive_items(*p->g, lp.layout);
      if (!alive.empty()) {
        o << ", \"alive_items\": [";
        bool first = true;
        for (size_t t = 0; t < alive.size(); t++)
          if (alive[t]) {
            o << (first ? "" : ", ") << t;
            first = false;
          }
        o << "]";
      }
    }
    // entries of the item list full-range counts hand out now (live items,
    // or the items and pieces of fbg_schedule_units)
    if (which == 0 && p->jb[0].valid && p->jb[0].d_perm) o << ", \"item_list_entries\": " << p->jb[0].nperm;
    o << "}";
  } else {
    InterpCode code;
    LutProgram lp;
    try {
      Layout L = make_layout(p->n, interp_params(p), order_for(p, which == 2));
      lp = lower_and_map(*p->g, L);
      if (!p->opt_prune) strip_prune(lp);
      code = emit_bytecode(lp);
    } catch (CompileError& e) {
      return set_error(FBG_ETOOBIG, e.msg);
    }
    const FbgInterpProg& G = code.prog;
    o << "{";
    layout_json(lp.layout);
    o << ", \"ins\": [";
    for (size_t i = 0; i < code.ins.size(); i++) o << (i ? ", " : "") << code.ins[i];
    o << "], \"consts\": [";
    for (size_t i = 0; i < code.consts.size(); i++) o << (i ? ", " : "") << code.consts[i];
    o << "], \"levels\": [";
    for (unsigned i = 0; i < G.nlevels; i++)
      o << (i ? ", " : "") << "[" << G.lev[i].ins_begin << ", " << G.lev[i].ins_end << ", " << G.lev[i].bits << ", "
        << G.lev[i].pos << ", " << G.lev[i].has_acc << ", " << G.lev[i].acc_op << "]";
    o << "], \"out_op\": " << G.out_op << ", \"nslots\": " << G.nslots << ", \"nshared\": " << G.nshared << ", \"tvalid\": " << G.tvalid
      << ", \"vmask\": " << G.vmask << ", \"first_unit_pos\": " << G.first_unit_pos << ", \"unit_bits\": "
      << G.unit_bits << ", \"nunits\": " << G.nunits;
    if (p->opt_prune) {   // units that a conjunct over unit and warp letters leaves alive (-1: not evaluated)
      const std::vector<uint64_t> alive = alive_words(*p->g, lp.layout);
      long long nlive = -1;
      if (!alive.empty()) {
        nlive = 0;
        const int wb = lp.layout.warp_bits;
        for (uint64_t u = 0; u < G.nunits; u++) {
          bool any = false;
          for (int w = 0; w < (1 << wb); w++) {
            const uint64_t t = (u << wb) | (uint64_t)w;
            any = any || ((alive[(size_t)(t >> 6)] >> (t & 63)) & 1);
          }
          nlive += any;
        }
      }
      o << ", \"live_units\": " << nlive;
    }
    o << "}";
  }
  std::string s = o.str();
  if (buf) {
    if (*len < s.size() + 1) return set_error(FBG_EINVAL, "buffer too small");
    std::memcpy(buf, s.c_str(), s.size() + 1);
  }
  *len = s.size() + 1;
  return FBG_OK;
}

fbg_status fbg_debug_nvrtc_compile(const char* body, char* log, size_t loglen) {
  if (!body) return set_error(FBG_EINVAL, "null argument");
  std::string lg;
  bool ok = jit_check(body, &lg);
  if (log && loglen) {
    size_t n = std::min(loglen - 1, lg.size());
    std::memcpy(log, lg.data(), n);
    log[n] = 0;
  }
  return ok ? FBG_OK : set_error(FBG_EJIT, lg);
}

const char* fbg_program_jit_log(fbg_program* p) { return p ? p->jit_log.c_str() : ""; }

void fbg_program_free(fbg_program* p) { delete p; }

const char* fbg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
