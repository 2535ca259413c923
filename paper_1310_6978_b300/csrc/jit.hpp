// jit.hpp -- NVRTC front end for the specialised kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace fbg {

struct JitResult {
  bool ok = false;
  bool cached = false;
  cudaKernel_t kernel = nullptr;
  std::string log;     // NVRTC / ptxas messages (registers, spills) or the error
};

// Compile fbg_device.cuh + body for sm_103a and load it on the current device.
JitResult jit_compile(const std::string& body, const char* kernel_name, int device);
size_t jit_cache_size();
// Kernels for many sources at once: a pool of worker threads compiles them
// (sources still compiling after deadline_s are not ok); each is loaded on
// this device and cached like jit_compile.
std::vector<JitResult> jit_compile_many(const std::vector<std::string>& bodies, const char* kernel_name, int device,
                                        double deadline_s, std::string* log);
// Compile only (no device needed); *log receives the NVRTC/ptxas messages.
bool jit_check(const std::string& body, std::string* log);
// Compile only, many sources on the pool of jit_compile_many (the same
// compiles and cache of compiled code a batch uses); per source whether it
// compiled before deadline_s.
std::vector<bool> jit_check_many(const std::vector<std::string>& bodies, double deadline_s, std::string* log);

}  // namespace fbg
