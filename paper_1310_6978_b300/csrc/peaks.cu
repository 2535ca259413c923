// peaks.cu -- the integer-logic roof of this GPU, measured: every thread runs
// 16 independent chains of lop3.b32 (no memory traffic, no dependencies
// between chains), so the SMs issue lop3 as fast as the ALU pipe allows.
// The rate is the denominator check for the count kernels' roofline.
#include <cuda_runtime.h>

#include <cstdint>

#include "fbg.h"
#include "fbg_device.cuh"

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) lop3_chains(uint32_t seed, int iters, uint32_t* sink) {
  uint32_t v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) v[c] = seed * (uint32_t)(c + 1) + threadIdx.x;
  const uint32_t a = seed ^ 0x9E3779B9u, b = seed + 0x7F4A7C15u;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = fbg_lop3<0x96>(v[c], a, b);   // xor3: no folding possible
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = fbg_lop3<0xe8>(v[c], b, a);   // majority
  }
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) x ^= v[c];
  if (x == 0x12345678u) sink[0] = x;   // keeps the chains alive
}

}  // namespace

extern "C" fbg_status fbg_probe_lop3_rate(void* stream, double* tops) {
  if (!tops) return FBG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FBG_ECUDA;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, 4) != cudaSuccess) return FBG_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  lop3_chains<<<blocks, threads, 0, st>>>(1u, 64, sink);   // warm-up
  cudaEventRecord(e0, st);
  lop3_chains<<<blocks, threads, 0, st>>>(2u, iters, sink);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return FBG_ECUDA;
  const double ops = (double)blocks * threads * iters * kChains * 2.0;
  *tops = ops / ((double)ms * 1e-3) / 1e12;
  return FBG_OK;
}
