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
// With FBG_BATCH_SPECIALIZE the distinct programs that carry most of the
// nominal work (each at least 1% of it, up to 16) are compiled by NVRTC into
// straight-line device functions inside ONE persistent batch kernel; the
// kernel's work-item loop calls a program's function when it has one and
// interprets its bytecode otherwise.  If that compilation fails the batch
// runs on the interpreter kernel alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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
    CKB(cudaLaunchKernel((const void*)b->kern, dim3((unsigned)b->grid), dim3(FBG_INTERP_BLOCK), args,
                         interp_smem_bytes(b->nslots), st));
  } else {
    CKB(launch_interp(0, b->d_progs, b->d_items, b->nitems, b->d_counts + np, b->d_counts, nullptr, P, b->nslots,
                      b->grid, st));
  }
  CKB(cudaMemcpyAsync(b->h_counts, b->d_counts, np * 8, cudaMemcpyDeviceToHost, st));
  return FBG_OK;
}

}  // namespace

// Choice of the programs to specialise and the source of the batch kernel
// (host only).  fid[i] receives program i's function id or -1.
std::string batch_kernel_source(fbg_program* const* progs, int nprogs, std::vector<int>& fid,
                                std::vector<LutProgram>& spec_lp, std::string* err) {
  fid.assign((size_t)nprogs, -1);
  spec_lp.clear();
  std::map<std::pair<std::string, int>, std::vector<int>> groups;
  double total_cost = 0;
  std::vector<double> cost((size_t)nprogs);
  for (int i = 0; i < nprogs; i++) {
    size_t ins = progs[i]->ib[0].valid ? progs[i]->ib[0].code.ins.size() : (size_t)progs[i]->g.dag.size();
    cost[(size_t)i] = std::ldexp((double)std::max<size_t>(1, ins), progs[i]->n);
    total_cost += cost[(size_t)i];
    groups[{progs[i]->text, progs[i]->k}].push_back(i);
  }
  std::vector<std::pair<double, const std::vector<int>*>> ranked;
  for (auto& g : groups) {
    double c = 0;
    for (int i : g.second) c += cost[(size_t)i];
    if (progs[g.second[0]]->n >= 13 && c >= 0.01 * total_cost) ranked.push_back({c, &g.second});
  }
  std::sort(ranked.begin(), ranked.end(), [](auto& x, auto& y) { return x.first > y.first; });
  if (ranked.size() > 16) ranked.resize(16);
  if (ranked.empty()) return "";
  std::string body = "#include \"interp_device.cuh\"\n";
  for (size_t gi = 0; gi < ranked.size(); gi++) {
    const fbg_program* p0 = progs[(*ranked[gi].second)[0]];
    LayoutParams lp;
    lp.r_max = 2;
    lp.warps_log2 = FBG_INTERP_WARPS_LOG2;   // the batch kernel's block shape
    lp.unit_bits_max = 13;
    lp.loop_level_bits = 2;
    try {
      Layout L = make_layout(p0->n, lp, search_order(p0->g));
      spec_lp.push_back(lower_and_map(p0->g, L));
      body += emit_batch_function(spec_lp.back(), "fbg_bp" + std::to_string(gi));
    } catch (CompileError& e) {
      if (err) *err = e.msg;
      fid.assign((size_t)nprogs, -1);
      spec_lp.clear();
      return "";
    }
    for (int i : *ranked[gi].second) fid[(size_t)i] = (int)gi;
  }
  body += "extern \"C\" __global__ void __launch_bounds__(" + std::to_string(FBG_INTERP_BLOCK) +
          ") fbg_batch_kernel(const FbgInterpProg* __restrict__ progs, const FbgWorkItem* __restrict__ items,"
          " fbg_u64 nitems, fbg_u64* item_ctr, fbg_u64* prog_counts, const int* __restrict__ fid) {\n"
          "  using namespace fbg_interp;\n"
          "  extern __shared__ fbg_u64 dyn_slots[];\n"
          "  __shared__ Shared S;\n"
          "  Thread T;\n"
          "  T.slots = dyn_slots + threadIdx.x;\n"
          "  T.acc = 0;\n"
          "  T.coords = 0;\n"
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
  for (size_t gi = 0; gi < spec_lp.size(); gi++)
    body += "      case " + std::to_string(gi) + ": cnt = fbg_bp" + std::to_string(gi) + "(W.unit_begin, W.unit_end, lvl); break;\n";
  body += "      default: process_item<0>(S, T, progs, W, cur, alive0, P, cnt, iters); break;\n"
          "    }\n"
          "    cnt = fbg_warp_sum(cnt);\n"
          "    if ((threadIdx.x & 31u) == 0u && cnt) atomicAdd(prog_counts + W.prog, cnt);\n"
          "  }\n"
          "}\n";
  return body;
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
    std::string body = batch_kernel_source(progs, nprogs, fid, spec_lp, &err);
    b->jit_log = err;
    if (!body.empty()) {
      int dev = 0;
      cudaGetDevice(&dev);
      JitResult r = jit_compile(body, "fbg_batch_kernel", dev);
      b->jit_log = r.log;
      if (r.ok) {
        b->kern = r.kernel;
        b->specialized = (int)spec_lp.size();
      } else {
        std::fill(fid.begin(), fid.end(), -1);
        spec_lp.clear();
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)b->kern, FBG_INTERP_BLOCK, smem) == cudaSuccess &&
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
  std::vector<int> fid;
  std::vector<LutProgram> spec_lp;
  std::string err;
  std::string src = batch_kernel_source(progs, nprogs, fid, spec_lp, &err);
  if (src.empty() && !err.empty()) return set_error(FBG_ETOOBIG, err);
  if (buf) {
    if (*len < src.size() + 1) return set_error(FBG_EINVAL, "buffer too small");
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  *len = src.size() + 1;
  return FBG_OK;
}

void fbg_batch_free(fbg_batch* b) { delete b; }

}  // extern "C"
