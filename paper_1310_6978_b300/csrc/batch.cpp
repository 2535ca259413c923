// batch.cpp -- many programs counted in one persistent launch.
//
// The counting procedure of Sec. 3.4 evaluates a whole family of reduced
// formulas; here any set of compiled programs is counted together.  Every
// program's unit range is cut into work items (program, unit range); the
// items are sorted by nominal cost (assignments x instructions), largest
// first, and blocks of the interpreter kernel pull them from a device
// counter, so large and small formulas share one launch without a tail of
// idle SMs.  Per-program partial counts are accumulated in device memory.
// With FBG_BATCH_GRAPH the memsets, the launch and the copy of the counts
// to pinned host memory are captured once in a CUDA graph and replayed.
//
// With FBG_BATCH_SPECIALIZE the distinct programs with n >= 20 that carry
// the most nominal work (up to 512) get straight-line device functions: each
// is compiled separately by NVRTC as relocatable device code (in parallel,
// cached per source), the dispatch kernel likewise, and nvJitLink links them
// into ONE persistent batch kernel whose work-item loop calls a program's
// function when it has one and interprets its bytecode otherwise.  Programs
// whose compilation fails or misses the deadline are interpreted; if the
// kernel itself cannot be built the batch runs on the interpreter kernel.
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

struct fbg_batch {
  std::vector<fbg_program*> progs;
  FbgInterpProg* d_progs = nullptr;
  FbgWorkItem* d_items = nullptr;
  unsigned long long* d_counts = nullptr;   // [nprogs] counts, then the item counter
  unsigned long long* h_counts = nullptr;   // pinned
  uint64_t nitems = 0, units = 0;
  unsigned nslots = 1;
  int grid = 1;
  bool use_graph = false;
  // specialised programs
  int specialized = 0;
  int* d_fid = nullptr;                     // per program: function id or -1
  std::vector<int> fid;
  cudaKernel_t kern = nullptr;              // hybrid kernel, or null: interpreter kernel
  std::string jit_log;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  ~fbg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_progs) cudaFree(d_progs);
    if (d_items) cudaFree(d_items);
    if (d_counts) cudaFree(d_counts);
    if (h_counts) cudaFreeHost(h_counts);
    if (d_fid) cudaFree(d_fid);
  }
};

#define CKB(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
  } while (0)

namespace {

fbg_status enqueue(fbg_batch* b, cudaStream_t st) {
  const size_t np = b->progs.size();
  CKB(cudaMemsetAsync(b->d_counts, 0, (np + 1) * 8, st));
  FbgLaunch P{};
  P.unit_begin = 0;
  P.unit_end = ~0ull;
  if (b->kern) {
    unsigned long long* item_ctr = b->d_counts + np;
    unsigned long long* counts = b->d_counts;
    const FbgInterpProg* progs = b->d_progs;
    const FbgWorkItem* items = b->d_items;
    unsigned long long nitems = b->nitems;
    const int* fid = b->d_fid;
    void* args[] = {(void*)&progs, (void*)&items, (void*)&nitems, (void*)&item_ctr, (void*)&counts, (void*)&fid};
    CKB(cudaLaunchKernel((const void*)b->kern, dim3((unsigned)b->grid), dim3(FBG_INTERP_THREADS), args,
                         interp_smem_bytes(b->nslots), st));
  } else {
    CKB(launch_interp(0, b->d_progs, b->d_items, b->nitems, b->d_counts + np, b->d_counts, nullptr, P, b->nslots,
                      b->grid, st));
  }
  CKB(cudaMemcpyAsync(b->h_counts, b->d_counts, np * 8, cudaMemcpyDeviceToHost, st));
  return FBG_OK;
}

}  // namespace

// at most this many distinct programs get a specialised function
constexpr size_t kMaxSpecialized = 512;
// specialised functions still compiling after this are dropped (interpreted)
constexpr double kCompileDeadlineS = 180.0;

struct BatchPlan {
  std::vector<int> fid;                 // per program: function id or -1
  std::vector<std::string> fn_name;     // per function
  std::vector<std::string> fn_src;      // per function (relocatable device code)
  std::vector<LutProgram> spec_lp;      // per function: its layout
};

// Choice of the programs to specialise (host only): distinct programs (by
// text and domain) with n >= 20, ranked by nominal work (instances x 2^n x
// program size), at most kMaxSpecialized.
BatchPlan plan_batch(fbg_program* const* progs, int nprogs, std::string* err) {
  BatchPlan plan;
  plan.fid.assign((size_t)nprogs, -1);
  std::map<std::pair<std::string, int>, std::vector<int>> groups;
  std::vector<double> cost((size_t)nprogs);
  for (int i = 0; i < nprogs; i++) {
    size_t ins = progs[i]->ib[0].valid ? progs[i]->ib[0].code.ins.size() : (size_t)progs[i]->g.dag.size();
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
    lp.warps_log2 = FBG_INTERP_WARPS_LOG2;   // the batch kernel's block shape
    lp.unit_bits_max = 13;
    lp.loop_level_bits = 2;
    char nm[64];
    std::snprintf(nm, sizeof nm, "fbg_bp_%016zx_%d", std::hash<std::string>()(p0->text), p0->k);
    try {
      Layout L = make_layout(p0->n, lp, search_order(p0->g));
      plan.spec_lp.push_back(lower_and_map(p0->g, L));
      plan.fn_src.push_back("extern \"C\" " + emit_batch_function(plan.spec_lp.back(), nm));
      plan.fn_name.push_back(nm);
    } catch (CompileError& e) {
      if (err) *err = e.msg;
      return BatchPlan{std::vector<int>((size_t)nprogs, -1), {}, {}, {}};
    }
    for (int i : *ranked[gi].second) plan.fid[(size_t)i] = (int)gi;
  }
  return plan;
}

// the persistent batch kernel: calls the specialised functions listed in
// `names` (by function id) and interprets every other program
std::string batch_kernel_source(const std::vector<std::string>& names) {
  std::string body = "#include \"interp_device.cuh\"\n";
  for (auto& nm : names) body += "extern \"C\" __device__ fbg_u64 " + nm + "(fbg_u64 u0, fbg_u64 u1, fbg_u32 tb, fbg_u64* lvl);\n";
  body += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(FBG_INTERP_THREADS) +
          ") fbg_batch_kernel(const FbgInterpProg* __restrict__ progs, const FbgWorkItem* __restrict__ items,"
          " fbg_u64 nitems, fbg_u64* item_ctr, fbg_u64* prog_counts, const int* __restrict__ fid) {\n"
          "  using namespace fbg_interp;\n"
          "  extern __shared__ fbg_u64 dyn_slots[];\n"
          "  __shared__ Shared S;\n"
          "  Thread T;\n"
          "  init_thread(T, dyn_slots);\n"
          "  unsigned cur = 0xFFFFFFFFu;\n"
          "  bool alive0 = true;\n"
          "  fbg_u64 iters = 0;\n"
          "  FbgLaunch P = {};\n"
          "  fbg_u64 lvl[16] = {0};\n"
          "  for (;;) {\n"
          "    if (threadIdx.x == 0) S.item = atomicAdd(item_ctr, 1ull);\n"
          "    __syncthreads();\n"
          "    const fbg_u64 item = S.item;\n"
          "    __syncthreads();\n"
          "    if (item >= nitems) break;\n"
          "    const FbgWorkItem W = items[item];\n"
          "    fbg_u64 cnt = 0;\n"
          "    switch (fid[W.prog]) {\n";
  for (size_t gi = 0; gi < names.size(); gi++)
    body += "      case " + std::to_string(gi) + ": cnt = " + names[gi] + "(W.unit_begin, W.unit_end, threadIdx.x, lvl) + " +
            names[gi] + "(W.unit_begin, W.unit_end, threadIdx.x + 32u, lvl); break;\n";
  body += "      default: process_item<0>(S, T, progs, W, cur, alive0, P, cnt, iters); break;\n"
          "    }\n"
          "    cnt = fbg_warp_sum(cnt);\n"
          "    if ((threadIdx.x & 31u) == 0u && cnt) atomicAdd(prog_counts + W.prog, cnt);\n"
          "  }\n"
          "}\n";
  return body;
}

// compile the plan's functions (in parallel) and the batch kernel; drops the
// functions that fail or miss the deadline; returns the relocatable cubins
bool build_batch_cubins(BatchPlan& plan, std::vector<std::string>* cubins, std::string* log) {
  std::vector<std::string> fn_cubins;
  std::vector<bool> ok = jit_compile_rdc_many(plan.fn_src, &fn_cubins, kCompileDeadlineS, log);
  std::vector<int> remap(plan.fn_src.size(), -1);
  std::vector<std::string> names;
  cubins->clear();
  cubins->push_back(std::string());   // the kernel, below
  std::vector<LutProgram> kept;
  for (size_t f = 0; f < ok.size(); f++) {
    if (!ok[f]) continue;
    remap[f] = (int)names.size();
    names.push_back(plan.fn_name[f]);
    cubins->push_back(fn_cubins[f]);
    kept.push_back(std::move(plan.spec_lp[f]));
  }
  for (auto& f : plan.fid) f = f >= 0 ? remap[(size_t)f] : -1;
  plan.spec_lp.swap(kept);
  plan.fn_name = names;
  std::vector<std::string> kc;
  std::string klog;
  std::vector<bool> kok = jit_compile_rdc_many({batch_kernel_source(names)}, &kc, kCompileDeadlineS, &klog);
  if (!kok[0]) {
    if (log) *log += klog;
    return false;
  }
  (*cubins)[0] = kc[0];
  return true;
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
  struct Item {
    FbgWorkItem w;
    double cost;
  };
  std::vector<Item> items;
  uint64_t total_units = 0;
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
    b->nslots = std::max(b->nslots, ib.code.nslots);
    total_units += ib.nunits;
  }
  // specialised functions for the distinct programs that carry the work
  std::vector<int> fid((size_t)nprogs, -1);
  std::vector<LutProgram> spec_lp;
  if (flags & FBG_BATCH_SPECIALIZE) {
    std::string err;
    BatchPlan plan = plan_batch(progs, nprogs, &err);
    b->jit_log = err;
    if (!plan.fn_src.empty()) {
      std::vector<std::string> cubins;
      if (build_batch_cubins(plan, &cubins, &b->jit_log)) {
        int dev = 0;
        cudaGetDevice(&dev);
        JitResult r = jit_link(cubins, "fbg_batch_kernel", dev);
        if (!r.log.empty()) b->jit_log += r.log;
        if (r.ok) {
          b->kern = r.kernel;
          b->specialized = (int)plan.fn_name.size();
          fid = plan.fid;
          spec_lp = std::move(plan.spec_lp);
        }
      }
    }
  }
  b->fid = fid;
  // units of each program in the layout its items are evaluated in
  std::vector<uint64_t> nunits((size_t)nprogs);
  total_units = 0;
  for (int i = 0; i < nprogs; i++) {
    nunits[(size_t)i] = fid[(size_t)i] >= 0 ? (1ull << spec_lp[(size_t)fid[(size_t)i]].layout.unit_bits)
                                              : progs[i]->ib[0].nunits;
    total_units += nunits[(size_t)i];
  }
  // item size: about 8 items per resident block, never more than max_item_units
  int per_sm = interp_blocks_per_sm(0, b->nslots);
  if (b->kern) {
    int dev = 0;
    cudaGetDevice(&dev);
    size_t smem = interp_smem_bytes(b->nslots);
    cudaKernelSetAttributeForDevice(b->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem, dev);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)b->kern, FBG_INTERP_THREADS, smem) == cudaSuccess &&
        nb > 0)
      per_sm = nb;
  }
  if (per_sm <= 0) {
    delete b;
    return set_error(FBG_ETOOBIG, "batch programs do not fit in shared memory");
  }
  uint64_t resident = (uint64_t)device_sms() * (uint64_t)per_sm;
  uint64_t target_items = resident * 8;
  uint64_t auto_units = std::max<uint64_t>(1, total_units / std::max<uint64_t>(1, target_items));
  uint64_t chunk = max_item_units ? max_item_units : auto_units;
  for (int i = 0; i < nprogs; i++) {
    const InterpBuild& ib = progs[i]->ib[0];
    uint64_t nu = nunits[(size_t)i];
    double unit_cost = (double)std::max<size_t>(1, ib.code.ins.size()) *
                       std::ldexp(1.0, progs[i]->n) / (double)nu;
    for (uint64_t u = 0; u < nu; u += chunk) {
      uint64_t e = std::min(nu, u + chunk);
      items.push_back(Item{FbgWorkItem{(unsigned)i, 0u, u, e}, unit_cost * (double)(e - u)});
    }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
  std::vector<FbgWorkItem> w;
  w.reserve(items.size());
  for (auto& it : items) w.push_back(it.w);
  b->nitems = w.size();
  b->units = total_units;
  b->grid = (int)std::min<uint64_t>(b->nitems, resident);
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_fid, (size_t)nprogs * sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpy(b->d_fid, fid.data(), (size_t)nprogs * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_progs, descs.size() * sizeof(FbgInterpProg))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_items, w.size() * sizeof(FbgWorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_counts, ((size_t)nprogs + 1) * 8)) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_counts, (size_t)nprogs * 8)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_progs, descs.data(), descs.size() * sizeof(FbgInterpProg), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(b->d_items, w.data(), w.size() * sizeof(FbgWorkItem), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete b;
    return cuda_error(e, "batch setup");
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
  if (plan.fn_src.empty() && !err.empty()) return set_error(FBG_ETOOBIG, err);
  std::string src = batch_kernel_source(plan.fn_name);
  for (auto& f : plan.fn_src) src += f;
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
  std::vector<std::string> cubins;
  bool ok = plan.fn_src.empty() || build_batch_cubins(plan, &cubins, &err);
  if (ok && !cubins.empty()) ok = jit_link_check(cubins, &err);
  if (specialized) *specialized = ok ? (int)plan.fn_name.size() : 0;
  if (log && loglen) {
    size_t n = std::min(loglen - 1, err.size());
    std::memcpy(log, err.data(), n);
    log[n] = 0;
  }
  return ok ? FBG_OK : set_error(FBG_EJIT, err);
}

void fbg_batch_free(fbg_batch* b) { delete b; }

}  // extern "C"
