// batch.cpp -- many programs counted in one persistent launch.
//
// The counting procedure of Sec. 3.4 evaluates a whole family of reduced
// formulas; here any set of compiled programs is counted together.  Every
// program's unit range is cut into work items (program, unit range); the
// items are sorted by nominal cost (assignments x instructions), largest
// first, and blocks of the interpreter kernel pull them from a device
// counter, so large and small formulas share one launch without a tail of
// idle SMs.  Per-program partial counts are accumulated in device memory.
// With use_graph the memsets, the launch and the copy of the counts to
// pinned host memory are captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fbg.h"
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
  CKB(launch_interp(0, b->d_progs, b->d_items, b->nitems, b->d_counts + np, b->d_counts, nullptr, P, b->nslots, b->grid,
                    st));
  CKB(cudaMemcpyAsync(b->h_counts, b->d_counts, np * 8, cudaMemcpyDeviceToHost, st));
  return FBG_OK;
}

}  // namespace

extern "C" {

fbg_status fbg_batch_create(fbg_program* const* progs, int nprogs, uint64_t max_item_units, int use_graph,
                            fbg_batch** out) {
  if (!progs || nprogs <= 0 || !out) return set_error(FBG_EINVAL, "bad argument");
  *out = nullptr;
  auto* b = new fbg_batch();
  b->progs.assign(progs, progs + nprogs);
  b->use_graph = use_graph != 0;
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
  // item size: about 8 items per resident block, never more than max_item_units
  int per_sm = interp_blocks_per_sm(0, b->nslots);
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
    uint64_t nu = ib.nunits;
    double unit_cost = (double)std::max<size_t>(1, ib.code.ins.size()) *
                       std::ldexp(1.0, progs[i]->n - (int)ib.lp.layout.unit_bits);
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
  if ((e = cudaMalloc(&b->d_progs, descs.size() * sizeof(FbgInterpProg))) != cudaSuccess ||
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

fbg_status fbg_batch_info(fbg_batch* b, uint64_t* items, uint64_t* units, int* grid) {
  if (!b) return set_error(FBG_EINVAL, "null batch");
  if (items) *items = b->nitems;
  if (units) *units = b->units;
  if (grid) *grid = b->grid;
  return FBG_OK;
}

void fbg_batch_free(fbg_batch* b) { delete b; }

}  // extern "C"
