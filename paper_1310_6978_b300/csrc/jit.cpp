// jit.cpp -- NVRTC compilation of specialised kernels for sm_103a and a
// process-wide cache keyed by the generated source, so identical programs
// (same formula, layout and mode) are compiled once.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "jit.hpp"

namespace fbg {

// device headers as text (generated by the build from the .cuh / .h files)
extern const char fbg_device_header[];
extern const char fbg_interp_format_header[];
extern const char fbg_interp_device_header[];

namespace {

struct Entry {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
};

std::mutex g_mu;
std::unordered_map<std::string, Entry> g_cache;   // key: device + source

}  // namespace

JitResult jit_compile(const std::string& body, const char* kernel_name, int device) {
  JitResult r;
  std::string src = "#include \"fbg_device.cuh\"\n" + body;
  std::string key = std::to_string(device) + ":" + kernel_name + ":" + src;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      r.ok = true;
      r.kernel = it->second.kern;
      r.cached = true;
      return r;
    }
  }
  // NVRTC runs on a worker thread with a time limit (FBG_JIT_TIMEOUT_S,
  // default 60 s): a compile that does not finish is abandoned (the thread
  // finishes on its own later) and the caller gets an error instead of a hang
  struct Job {
    std::mutex mu;
    std::condition_variable cv;
    bool done = false, ok = false;
    std::string cubin, log;
  };
  auto job = std::make_shared<Job>();
  std::thread([job, src] {
    std::string cubin, log;
    bool ok = false;
    const char* hdrs[3] = {fbg_device_header, fbg_interp_format_header, fbg_interp_device_header};
    const char* names[3] = {"fbg_device.cuh", "interp_format.h", "interp_device.cuh"};
    nvrtcProgram prog;
    nvrtcResult e = nvrtcCreateProgram(&prog, src.c_str(), "fbg_jit.cu", 3, hdrs, names);
    if (e != NVRTC_SUCCESS) {
      log = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(e);
    } else {
      const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
      e = nvrtcCompileProgram(prog, 4, opts);
      size_t logn = 0;
      nvrtcGetProgramLogSize(prog, &logn);
      if (logn > 1) {
        log.resize(logn);
        nvrtcGetProgramLog(prog, &log[0]);
        while (!log.empty() && (log.back() == 0 || log.back() == '\n')) log.pop_back();
      }
      if (e != NVRTC_SUCCESS) {
        log = std::string("nvrtcCompileProgram: ") + nvrtcGetErrorString(e) + "\n" + log;
      } else {
        size_t n = 0;
        nvrtcGetCUBINSize(prog, &n);
        cubin.assign(n, '\0');
        nvrtcGetCUBIN(prog, &cubin[0]);
        ok = true;
      }
      nvrtcDestroyProgram(&prog);
    }
    std::lock_guard<std::mutex> lk(job->mu);
    job->cubin = std::move(cubin);
    job->log = std::move(log);
    job->ok = ok;
    job->done = true;
    job->cv.notify_all();
  }).detach();
  double limit = 60.0;
  if (const char* env = std::getenv("FBG_JIT_TIMEOUT_S")) limit = std::atof(env) > 0 ? std::atof(env) : limit;
  std::string cubin;
  {
    std::unique_lock<std::mutex> lk(job->mu);
    if (!job->cv.wait_for(lk, std::chrono::duration<double>(limit), [&] { return job->done; })) {
      r.log = "NVRTC compilation exceeded " + std::to_string((int)limit) + " s and was abandoned";
      return r;
    }
    r.log = job->log;
    if (!job->ok) return r;
    cubin = job->cubin;
  }
  Entry ent;
  cudaError_t ce = cudaLibraryLoadData(&ent.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (ce != cudaSuccess) {
    r.log = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(ce);
    return r;
  }
  ce = cudaLibraryGetKernel(&ent.kern, ent.lib, kernel_name);
  if (ce != cudaSuccess) {
    r.log = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(ce);
    cudaLibraryUnload(ent.lib);
    return r;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto ins = g_cache.emplace(key, ent);
    if (!ins.second) {
      cudaLibraryUnload(ent.lib);
      ent = ins.first->second;
    }
  }
  r.ok = true;
  r.kernel = ent.kern;
  return r;
}

bool jit_check(const std::string& body, std::string* log) {
  std::string src = "#include \"fbg_device.cuh\"\n" + body;
  const char* hdrs[3] = {fbg_device_header, fbg_interp_format_header, fbg_interp_device_header};
  const char* names[3] = {"fbg_device.cuh", "interp_format.h", "interp_device.cuh"};
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "fbg_jit.cu", 3, hdrs, names) != NVRTC_SUCCESS) return false;
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
  nvrtcResult e = nvrtcCompileProgram(prog, 4, opts);
  size_t logn = 0;
  nvrtcGetProgramLogSize(prog, &logn);
  if (log && logn > 1) {
    log->resize(logn);
    nvrtcGetProgramLog(prog, &(*log)[0]);
  }
  nvrtcDestroyProgram(&prog);
  return e == NVRTC_SUCCESS;
}

size_t jit_cache_size() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_cache.size();
}

}  // namespace fbg
