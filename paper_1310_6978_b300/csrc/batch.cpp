// batch.cpp -- many programs counted together.
//
// The counting procedure of Sec. 3.4 evaluates a whole family of reduced
// formulas; here any set of compiled programs is counted together.
//
// Interpreted programs: every program's unit range is cut into work items
// (program, unit range); the items are sorted by nominal cost (assignments x
// instructions), largest first, and the warps of ONE interpreter launch pull
// them from a device counter, so large and small formulas share the launch
// without a tail of idle SMs.  Per-program counts accumulate in device memory.
//
// With FBG_BATCH_SPECIALIZE the distinct programs with n >= 20 that carry the
// most nominal work (up to 512) get their own specialised count kernel (the
// one a single program uses, built by NVRTC in parallel, cached per source).
// Each instance of such a program is one launch of its kernel with its own
// four counter words (self-resetting: no memset between runs); the launches
// are spread over eight side streams longest first, by a time measured once
// per kernel when the batch is created, and the interpreter launch takes a
// stream of its own, so short kernels fill the SMs that long ones leave idle.
// Programs whose compilation fails or misses the deadline are interpreted.
//
// With FBG_BATCH_GRAPH the memset, the fork, all launches, the join and the
// copy of the counts to pinned host memory are captured once in a CUDA graph
// and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fbg.h"
#include "emit.hpp"
#include "jit.hpp"
#include "kernels.hpp"
#include "program.hpp"

using namespace fbg;

namespace {

// a specialised count kernel shared by the instances of one distinct program
struct SpecKernel {
  cudaKernel_t kern = nullptr;
  int grid = 1, block = 32;
  uint64_t nunits = 1, chunk = 1;
  unsigned nwarps = 1;
  unsigned* d_items = nullptr;   // live (unit, slice) items, or null: all
  uint64_t nitems = 0;
  float ms = 0.f;   // one launch, measured when the batch is created
};

constexpr int kSideStreams = 8;
constexpr size_t kInstWords = 4;   // item counter, running sum, finished warps, pad

}  // namespace

struct fbg_batch {
  std::vector<fbg_program*> progs;
  FbgInterpProg* d_progs = nullptr;
  FbgWorkItem* d_items = nullptr;
  unsigned long long* d_counts = nullptr;   // [nprogs] counts, then the interpreter's item counter
  unsigned long long* h_counts = nullptr;   // pinned
  uint64_t nitems = 0, units = 0;
  unsigned nslots = 1;
  int grid = 1;
  bool use_graph = false;
  // specialised programs
  int specialized = 0;
  std::vector<int> fid;                     // per program: kernel id or -1
  std::vector<SpecKernel> spec;
  unsigned long long* d_inst = nullptr;     // kInstWords counter words per program
  std::vector<std::vector<int>> lanes;      // per side stream: the programs launched there
  std::vector<cudaStream_t> side;           // side streams (kSideStreams + 1 for the interpreter)
  std::vector<cudaEvent_t> ev;              // fork + one join event per side stream
  std::string jit_log;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~fbg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    if (d_progs) cudaFree(d_progs);
    if (d_items) cudaFree(d_items);
    if (d_counts) cudaFree(d_counts);
    if (h_counts) cudaFreeHost(h_counts);
    if (d_inst) cudaFree(d_inst);
    for (SpecKernel& k : spec)
      if (k.d_items) cudaFree(k.d_items);
  }
};

#define CKB(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
  } while (0)

namespace {

// one self-resetting launch of a specialised kernel for program i
cudaError_t launch_spec(const fbg_batch* b, int i, cudaStream_t st) {
  const SpecKernel& k = b->spec[(size_t)b->fid[(size_t)i]];
  unsigned long long* w = b->d_inst + (size_t)i * kInstWords;
  FbgLaunch P{};
  P.unit_ctr = w + 0;
  P.acc = w + 1;
  P.done = w + 2;
  P.out = b->d_counts + i;
  P.nwarps = k.nwarps;
  P.unit_begin = 0;
  P.unit_end = k.nunits;
  P.chunk = k.chunk;
  if (k.d_items) {
    P.unit_perm = k.d_items;
    P.nperm = k.nitems;
  }
  void* args[] = {&P};
  return cudaLaunchKernel((const void*)k.kern, dim3((unsigned)k.grid), dim3((unsigned)k.block), args, 0, st);
}

fbg_status enqueue(fbg_batch* b, cudaStream_t st) {
  const size_t np = b->progs.size();
  CKB(cudaMemsetAsync(b->d_counts, 0, (np + 1) * 8, st));
  FbgLaunch P{};
  P.unit_begin = 0;
  P.unit_end = ~0ull;
  if (b->side.empty()) {
    if (b->nitems)
      CKB(launch_interp(0, b->d_progs, b->d_items, b->nitems, b->d_counts + np, b->d_counts, nullptr, P, b->nslots,
                        b->grid, st));
  } else {
    // fork: every side stream waits for the memset
    CKB(cudaEventRecord(b->ev[0], st));
    for (size_t s = 0; s < b->side.size(); s++) CKB(cudaStreamWaitEvent(b->side[s], b->ev[0], 0));
    cudaStream_t is = b->side.back();
    if (b->nitems)
      CKB(launch_interp(0, b->d_progs, b->d_items, b->nitems, b->d_counts + np, b->d_counts, nullptr, P, b->nslots,
                        b->grid, is));
    for (size_t s = 0; s < b->lanes.size(); s++)
      for (int i : b->lanes[s]) CKB(launch_spec(b, i, b->side[s]));
    // join
    for (size_t s = 0; s < b->side.size(); s++) {
      CKB(cudaEventRecord(b->ev[s + 1], b->side[s]));
      CKB(cudaStreamWaitEvent(st, b->ev[s + 1], 0));
    }
  }
  CKB(cudaMemcpyAsync(b->h_counts, b->d_counts, np * 8, cudaMemcpyDeviceToHost, st));
  return FBG_OK;
}

}  // namespace

// at most this many distinct programs get a specialised kernel
constexpr size_t kMaxSpecialized = 512;
// specialised kernels still compiling after this are dropped (interpreted)
constexpr double kCompileDeadlineS = 180.0;

struct BatchPlan {
  std::vector<int> fid;                 // per program: kernel id or -1
  std::vector<std::string> src;         // per kernel: complete NVRTC source
  std::vector<LutProgram> lp;           // per kernel: its layout and LUTs
  std::vector<int> block;               // per kernel: threads per block
  std::vector<std::vector<unsigned>> live;   // per kernel: live items (when filtered)
  std::vector<char> filtered;                 // per kernel: 1 = hand out `live` only
};

// Choice of the programs to specialise (host only): distinct programs (by
// text and domain) with n >= 20, ranked by nominal work (instances x 2^n x
// program size), at most kMaxSpecialized; each gets the count kernel of a
// single program (4 warps per block, 4 words per thread, 2-bit loop levels).
BatchPlan plan_batch(fbg_program* const* progs, int nprogs, std::string* err) {
  BatchPlan plan;
  plan.fid.assign((size_t)nprogs, -1);
  std::map<std::pair<std::string, int>, std::vector<int>> groups;
  std::vector<double> cost((size_t)nprogs);
  for (int i = 0; i < nprogs; i++) {
    size_t ins = progs[i]->ib[0].valid ? progs[i]->ib[0].code.ins.size() : (size_t)progs[i]->g->dag.size();
    cost[(size_t)i] = std::ldexp((double)std::max<size_t>(1, ins), progs[i]->n);
    groups[{progs[i]->text, progs[i]->k}].push_back(i);
  }
  std::vector<std::pair<double, const std::vector<int>*>> ranked;
  for (auto& g : groups) {
    double c = 0;
    for (int i : g.second) c += cost[(size_t)i];
    if (progs[g.second[0]]->n >= 20) ranked.push_back({c, &g.second});
  }
  std::sort(ranked.begin(), ranked.end(), [](auto& x, auto& y) { return x.first > y.first; });
  if (ranked.size() > kMaxSpecialized) ranked.resize(kMaxSpecialized);
  for (size_t gi = 0; gi < ranked.size(); gi++) {
    const fbg_program* p0 = progs[(*ranked[gi].second)[0]];
    LayoutParams lp;
    lp.r_max = 2;
    lp.warps_log2 = 2;
    lp.unit_bits_max = 13;
    lp.loop_level_bits = 2;
    try {
      Layout L = make_layout(p0->n, lp, search_order(*p0->g));
      LutProgram prog = lower_and_map(*p0->g, L);
      int block = prog.layout.lane_bits < 5 ? 32 : 32 << prog.layout.warp_bits;
      plan.src.push_back(emit_cuda_source(prog, 0, block, 2, nullptr, nullptr, false));
      plan.block.push_back(block);
      // units whose unit-only conjuncts are false have no models: left out
      // when that removes at least a quarter of them
      std::vector<uint8_t> alive = alive_items(*p0->g, prog.layout);
      std::vector<unsigned> live;
      uint64_t nlive = 0;
      for (uint8_t a : alive) nlive += a;
      const bool filter = !alive.empty() && nlive * 4 <= alive.size() * 3;
      if (filter)
        for (size_t t = 0; t < alive.size(); t++)
          if (alive[t]) live.push_back((unsigned)t);
      plan.live.push_back(std::move(live));
      plan.filtered.push_back(filter ? 1 : 0);
      plan.lp.push_back(std::move(prog));
    } catch (CompileError& e) {
      if (err) *err = e.msg;
      return BatchPlan{std::vector<int>((size_t)nprogs, -1), {}, {}, {}, {}, {}};
    }
    for (int i : *ranked[gi].second) plan.fid[(size_t)i] = (int)gi;
  }
  return plan;
}

extern "C" {

fbg_status fbg_batch_create(fbg_program* const* progs, int nprogs, uint64_t max_item_units, int flags,
                            fbg_batch** out) {
  if (!progs || nprogs <= 0 || !out) return set_error(FBG_EINVAL, "bad argument");
  *out = nullptr;
  auto* b = new fbg_batch();
  b->progs.assign(progs, progs + nprogs);
  b->use_graph = (flags & FBG_BATCH_GRAPH) != 0;
  std::vector<FbgInterpProg> descs((size_t)nprogs);
  for (int i = 0; i < nprogs; i++) {
    fbg_program* p = progs[i];
    if (!p) {
      delete b;
      return set_error(FBG_EINVAL, "null program in batch");
    }
    if (p->n > 63) {
      delete b;
      return set_error(FBG_ETOOBIG, "counts need n <= 63");
    }
    fbg_status s = build_interp(p, 0);
    if (s != FBG_OK) {
      delete b;
      return s;
    }
    const InterpBuild& ib = p->ib[0];
    FbgInterpProg G = ib.code.prog;
    G.ins = ib.d_ins;
    G.consts = ib.d_consts;
    descs[(size_t)i] = G;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  // specialised kernels for the distinct programs that carry the work
  b->fid.assign((size_t)nprogs, -1);
  if (flags & FBG_BATCH_SPECIALIZE) {
    std::string err;
    BatchPlan plan = plan_batch(progs, nprogs, &err);
    b->jit_log = err;
    std::vector<JitResult> built = jit_compile_many(plan.src, "fbg_jit_count", dev, kCompileDeadlineS, &b->jit_log);
    std::vector<int> remap(plan.src.size(), -1);
    for (size_t k = 0; k < built.size(); k++) {
      if (!built[k].ok) continue;
      SpecKernel sk;
      sk.kern = built[k].kernel;
      sk.block = plan.block[k];
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)sk.kern, sk.block, 0) != cudaSuccess ||
          per_sm <= 0)
        per_sm = 1;
      sk.nunits = 1ull << plan.lp[k].layout.unit_bits;
      sk.grid = (int)std::min<uint64_t>(sk.nunits, (uint64_t)device_sms() * (uint64_t)per_sm);
      sk.chunk = std::max<uint64_t>(1, sk.nunits / ((uint64_t)sk.grid * 16));
      sk.nwarps = (unsigned)((uint64_t)sk.grid * (uint64_t)sk.block / 32);
      const std::vector<unsigned>& live = plan.live[k];
      if (plan.filtered[k]) {
        // live items only (possibly none); on failure all items run
        if (cudaMalloc(&sk.d_items, std::max<size_t>(1, live.size()) * sizeof(unsigned)) == cudaSuccess &&
            (live.empty() || cudaMemcpy(sk.d_items, live.data(), live.size() * sizeof(unsigned),
                                        cudaMemcpyHostToDevice) == cudaSuccess)) {
          sk.nitems = live.size();
          // only the blocks a short list needs
          const uint64_t wpb = (uint64_t)(sk.block / 32);
          sk.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sk.grid, (sk.nitems + wpb - 1) / wpb));
          sk.nwarps = (unsigned)((uint64_t)sk.grid * wpb);
          sk.chunk = std::max<uint64_t>(1, sk.nitems / ((uint64_t)sk.nwarps * 16));
        } else if (sk.d_items) {
          cudaFree(sk.d_items);
          sk.d_items = nullptr;
        }
      }
      remap[k] = (int)b->spec.size();
      b->spec.push_back(sk);
    }
    for (int i = 0; i < nprogs; i++)
      if (plan.fid[(size_t)i] >= 0) b->fid[(size_t)i] = remap[(size_t)plan.fid[(size_t)i]];
    b->specialized = (int)b->spec.size();
  }
  // interpreter items for the other programs
  struct Item {
    FbgWorkItem w;
    double cost;
  };
  std::vector<Item> items;
  uint64_t interp_units = 0, total_units = 0;
  for (int i = 0; i < nprogs; i++) {
    const int f = b->fid[(size_t)i];
    if (f >= 0) {
      total_units += b->spec[(size_t)f].nunits;
    } else {
      b->nslots = std::max(b->nslots, progs[i]->ib[0].code.nslots);
      interp_units += progs[i]->ib[0].live_units();
    }
  }
  total_units += interp_units;
  int per_sm = interp_blocks_per_sm(0, b->nslots);
  if (per_sm <= 0) {
    delete b;
    return set_error(FBG_ETOOBIG, "batch programs do not fit in shared memory");
  }
  // item size: about 8 items per resident block, never more than max_item_units
  uint64_t resident = (uint64_t)device_sms() * (uint64_t)per_sm;
  uint64_t target_items = resident * 8;
  uint64_t auto_units = std::max<uint64_t>(1, interp_units / std::max<uint64_t>(1, target_items));
  uint64_t chunk = max_item_units ? max_item_units : auto_units;
  for (int i = 0; i < nprogs; i++) {
    if (b->fid[(size_t)i] >= 0) continue;
    const InterpBuild& ib = progs[i]->ib[0];
    double unit_cost = (double)std::max<size_t>(1, ib.code.ins.size()) * std::ldexp(1.0, progs[i]->n) / (double)ib.nunits;
    // runs of live units (all units when none was left out), at most `chunk` each
    std::vector<FbgWorkItem> runs;
    if (ib.units_per_item == 1) {
      ib.append_items(runs, (unsigned)i, 0, ib.live_units(), chunk);
    } else {
      for (uint64_t u = 0; u < ib.nunits; u += chunk)
        runs.push_back(FbgWorkItem{(unsigned)i, 0u, u, std::min(ib.nunits, u + chunk)});
    }
    for (const FbgWorkItem& r : runs) items.push_back(Item{r, unit_cost * (double)(r.unit_end - r.unit_begin)});
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
  std::vector<FbgWorkItem> w;
  w.reserve(items.size());
  for (auto& it : items) w.push_back(it.w);
  b->nitems = w.size();
  b->units = total_units;
  b->grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(b->nitems, resident));
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_progs, descs.size() * sizeof(FbgInterpProg))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_items, std::max<size_t>(1, w.size()) * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_counts, ((size_t)nprogs + 1) * 8)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_counts, (size_t)nprogs * 8)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_inst, (size_t)nprogs * kInstWords * 8)) != cudaSuccess ||
      (e = cudaMemset(b->d_inst, 0, (size_t)nprogs * kInstWords * 8)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_progs, descs.data(), descs.size() * sizeof(FbgInterpProg), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (w.size() && (e = cudaMemcpy(b->d_items, w.data(), w.size() * sizeof(FbgWorkItem), cudaMemcpyHostToDevice)) !=
                       cudaSuccess)) {
    delete b;
    return cuda_error(e, "batch setup");
  }
  if (!b->spec.empty()) {
    // one timed launch per kernel (after one untimed), on a private stream
    cudaStream_t ts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<int> first(b->spec.size(), -1);
    for (int i = 0; i < nprogs; i++)
      if (b->fid[(size_t)i] >= 0 && first[(size_t)b->fid[(size_t)i]] < 0) first[(size_t)b->fid[(size_t)i]] = i;
    e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (size_t k = 0; k < b->spec.size() && e == cudaSuccess; k++) {
      e = launch_spec(b, first[k], ts);
      if (e == cudaSuccess) e = cudaEventRecord(e0, ts);
      if (e == cudaSuccess) e = launch_spec(b, first[k], ts);
      if (e == cudaSuccess) e = cudaEventRecord(e1, ts);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b->spec[k].ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ts) cudaStreamDestroy(ts);
    if (e != cudaSuccess) {
      delete b;
      return cuda_error(e, "batch kernel timing");
    }
    // longest processing time first over the side streams
    std::vector<int> order;
    for (int i = 0; i < nprogs; i++)
      if (b->fid[(size_t)i] >= 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return b->spec[(size_t)b->fid[(size_t)x]].ms > b->spec[(size_t)b->fid[(size_t)y]].ms;
    });
    b->lanes.assign(kSideStreams, {});
    std::vector<double> load(kSideStreams, 0.0);
    for (int i : order) {
      size_t s = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
      b->lanes[s].push_back(i);
      load[s] += b->spec[(size_t)b->fid[(size_t)i]].ms;
    }
    b->side.assign(kSideStreams + 1, nullptr);
    b->ev.assign(kSideStreams + 2, nullptr);
    for (auto& s : b->side)
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (auto& ev : b->ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      delete b;
      return cuda_error(e, "batch streams");
    }
  }
  *out = b;
  return FBG_OK;
}

fbg_status fbg_batch_run(fbg_batch* b, void* stream) {
  if (!b) return set_error(FBG_EINVAL, "null batch");
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->use_graph) return enqueue(b, st);
  if (!b->exec) {
    // capture on a private stream, then launch on the caller's stream
    cudaStream_t cap;
    CKB(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_error(e, "cudaStreamBeginCapture");
    }
    fbg_status s = enqueue(b, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (s != FBG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    b->graph = g;
    CKB(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  CKB(cudaGraphLaunch(b->exec, st));
  return FBG_OK;
}

fbg_status fbg_batch_results(fbg_batch* b, void* stream, uint64_t* host_counts) {
  if (!b || !host_counts) return set_error(FBG_EINVAL, "null argument");
  CKB(cudaStreamSynchronize((cudaStream_t)stream));
  std::memcpy(host_counts, b->h_counts, b->progs.size() * 8);
  return FBG_OK;
}

fbg_status fbg_batch_info(fbg_batch* b, uint64_t* items, uint64_t* units, int* grid, int* specialized) {
  if (!b) return set_error(FBG_EINVAL, "null batch");
  if (specialized) *specialized = b->specialized;
  if (items) *items = b->nitems;
  if (units) *units = b->units;
  if (grid) *grid = b->grid;
  return FBG_OK;
}

fbg_status fbg_batch_program_kinds(fbg_batch* b, int* specialized) {
  if (!b || !specialized) return set_error(FBG_EINVAL, "null argument");
  for (size_t i = 0; i < b->fid.size(); i++) specialized[i] = b->fid[i] >= 0 ? 1 : 0;
  return FBG_OK;
}

fbg_status fbg_debug_batch_source(fbg_program* const* progs, int nprogs, char* buf, size_t* len) {
  if (!progs || nprogs <= 0 || !len) return set_error(FBG_EINVAL, "bad argument");
  std::string err;
  BatchPlan plan = plan_batch(progs, nprogs, &err);
  if (plan.src.empty() && !err.empty()) return set_error(FBG_ETOOBIG, err);
  std::string src;
  for (size_t k = 0; k < plan.src.size(); k++) src += "// specialised count kernel " + std::to_string(k) + "\n" + plan.src[k];
  if (buf) {
    if (*len < src.size() + 1) return set_error(FBG_EINVAL, "buffer too small");
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  *len = src.size() + 1;
  return FBG_OK;
}

fbg_status fbg_debug_batch_build(fbg_program* const* progs, int nprogs, int* specialized, char* log, size_t loglen) {
  if (!progs || nprogs <= 0) return set_error(FBG_EINVAL, "bad argument");
  std::string err;
  BatchPlan plan = plan_batch(progs, nprogs, &err);
  // the compiles of fbg_batch_create, on its pool of worker threads
  std::string lg;
  const std::vector<bool> built = jit_check_many(plan.src, kCompileDeadlineS, &lg);
  int good = 0;
  for (bool b : built) good += b ? 1 : 0;
  const bool ok = good == (int)built.size();
  if (!ok && err.size() < 4096) err += lg;
  if (specialized) *specialized = good;
  if (log && loglen) {
    size_t n = std::min(loglen - 1, err.size());
    std::memcpy(log, err.data(), n);
    log[n] = 0;
  }
  return ok ? FBG_OK : set_error(FBG_EJIT, err);
}

void fbg_batch_free(fbg_batch* b) { delete b; }

}  // extern "C"
