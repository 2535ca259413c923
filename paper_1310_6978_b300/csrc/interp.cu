// interp.cu -- generic bytecode interpreter kernels (sm_103a).
//
// Evaluates any compiled program without a JIT (device code in
// interp_device.cuh).  One kernel serves single programs and the persistent
// batch: blocks pull work items (program, unit range) from a device counter.
#include <cuda_runtime.h>

#include <mutex>

#include "interp_device.cuh"
#include "kernels.hpp"

namespace fbg {

using namespace fbg_interp;

namespace {

template <int MODE>
__global__ void __launch_bounds__(NT) interp_kernel(const FbgInterpProg* __restrict__ progs,
                                                   const FbgWorkItem* __restrict__ items, fbg_u64 nitems,
                                                   fbg_u64* item_ctr, fbg_u64* prog_counts, fbg_u64* unit_counts,
                                                   FbgLaunch P, const FbgSlotOut* __restrict__ slot_out) {
  extern __shared__ __align__(16) fbg_u64 dyn_slots[];
  __shared__ Shared S;
  Thread T;
  init_thread(T, dyn_slots);
  unsigned cur = 0xFFFFFFFFu;
  bool alive0 = true;
  if (P.iters && threadIdx.x == 0)
    for (int lv = 0; lv < FBG_INTERP_MAX_LEVELS; lv++) S.lev_iters[lv] = 0;
  for (;;) {
    if (threadIdx.x == 0) S.item = atomicAdd(item_ctr, 1ull);
    __syncthreads();
    fbg_u64 item = S.item;
    __syncthreads();
    if (item >= nitems) break;
    FbgWorkItem W = items[item];
    fbg_u64 cnt = 0;
    if (MODE == 2 && slot_out) {
      // the program's own offsets, model buffer and capacity
      FbgLaunch Q = P;
      const FbgSlotOut so = slot_out[W.prog];
      Q.unit_begin = 0;
      Q.unit_offsets = so.unit_offsets;
      Q.models = so.models;
      Q.cap = so.cap;
      process_item<MODE>(S, T, progs, W, cur, alive0, Q, cnt);
    } else {
      process_item<MODE>(S, T, progs, W, cur, alive0, P, cnt);
    }
    if (MODE == 0) {
      cnt = fbg_warp_sum(cnt);
      if ((threadIdx.x & 31) == 0 && cnt) {
        if (prog_counts) atomicAdd(prog_counts + W.prog, cnt);
        // per-unit counts: items of one unit each (the caller ensures it)
        if (unit_counts) atomicAdd(unit_counts + (W.unit_begin - P.unit_begin), cnt);
        if (slot_out && (W.flags & FBG_ITEM_UNIT_COUNTS)) atomicAdd(slot_out[W.prog].unit_counts + W.unit_begin, cnt);
      }
    }
  }
  if (P.iters && threadIdx.x == 0)
    for (int lv = 0; lv < FBG_INTERP_MAX_LEVELS; lv++)
      if (S.lev_iters[lv]) atomicAdd(P.iters + lv, S.lev_iters[lv]);
}

// exclusive prefix sum of n u64 values, one block; total -> *total
__global__ void scan_kernel(const fbg_u64* in, fbg_u64* out, fbg_u64 n, fbg_u64* total) {
  __shared__ fbg_u64 part[1024];
  const unsigned t = threadIdx.x;
  fbg_u64 per = (n + 1023) / 1024;
  fbg_u64 lo = t * per, hi = lo + per < n ? lo + per : n;
  fbg_u64 s = 0;
  for (fbg_u64 i = lo; i < hi; i++) s += in[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    fbg_u64 run = 0;
    for (int i = 0; i < 1024; i++) {
      fbg_u64 v = part[i];
      part[i] = run;
      run += v;
    }
    if (total) *total = run;
  }
  __syncthreads();
  fbg_u64 run = part[t];
  for (fbg_u64 i = lo; i < hi; i++) {
    fbg_u64 v = in[i];
    out[i] = run;
    run += v;
  }
}

// out[i] = value for i < n (grid-stride)
__global__ void fill_u64_kernel(fbg_u64* out, fbg_u64 n, fbg_u64 value) {
  for (fbg_u64 i = (fbg_u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (fbg_u64)gridDim.x * blockDim.x)
    out[i] = value;
}

}  // namespace

size_t interp_smem_bytes(unsigned nslots) { return (size_t)nslots * B * sizeof(fbg_u64); }

// the dynamic shared memory limit is raised only when a larger size is needed,
// so launches (also inside stream capture) do not call cudaFuncSetAttribute;
// the attribute belongs to the current device, so the size set is kept per
// device (up to 64 devices; others set the attribute on every call)
static cudaError_t ensure_smem(int mode, size_t smem) {
  static std::mutex mu;
  static size_t set_to[64][3] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < 64;
  std::lock_guard<std::mutex> lock(mu);
  if (cached && smem <= set_to[dev][mode]) return cudaSuccess;
  if (mode == 0) e = cudaFuncSetAttribute(interp_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if (mode == 1) e = cudaFuncSetAttribute(interp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else e = cudaFuncSetAttribute(interp_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cached) set_to[dev][mode] = smem;
  return e;
}

cudaError_t launch_interp(int mode, const FbgInterpProg* progs, const FbgWorkItem* items, unsigned long long nitems,
                          unsigned long long* item_ctr, unsigned long long* prog_counts,
                          unsigned long long* unit_counts, const FbgLaunch& P, unsigned nslots, int grid,
                          cudaStream_t stream, const FbgSlotOut* slot_out) {
  size_t smem = interp_smem_bytes(nslots);
  cudaError_t e = ensure_smem(mode, smem);
  if (e != cudaSuccess) return e;
  if (mode == 0)
    interp_kernel<0><<<grid, NT, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, unit_counts, P, slot_out);
  else if (mode == 1)
    interp_kernel<1><<<grid, NT, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, unit_counts, P, slot_out);
  else
    interp_kernel<2><<<grid, NT, smem, stream>>>(progs, items, nitems, item_ctr, prog_counts, unit_counts, P, slot_out);
  return cudaGetLastError();
}

cudaError_t launch_scan(const unsigned long long* in, unsigned long long* out, unsigned long long n,
                        unsigned long long* total, cudaStream_t stream) {
  scan_kernel<<<1, 1024, 0, stream>>>(in, out, n, total);
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long* out, unsigned long long n, unsigned long long value,
                            cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const unsigned long long blocks = (n + 255) / 256;
  fill_u64_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, stream>>>(out, n, value);
  return cudaGetLastError();
}

int interp_blocks_per_sm(int mode, unsigned nslots) {
  int nb = 0;
  size_t smem = interp_smem_bytes(nslots);
  if (ensure_smem(mode, smem) != cudaSuccess) return 0;
  if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<0>, NT, smem);
  else if (mode == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<1>, NT, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, interp_kernel<2>, NT, smem);
  return nb;
}

}  // namespace fbg
