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
#include <vector>

#include "jit.hpp"

namespace fbg {

// device headers as text (generated by the build from the .cuh / .h files)
extern const char fbg_device_header[];

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
    const char* hdrs[1] = {fbg_device_header};
    const char* names[1] = {"fbg_device.cuh"};
    nvrtcProgram prog;
    nvrtcResult e = nvrtcCreateProgram(&prog, src.c_str(), "fbg_jit.cu", 1, hdrs, names);
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
  const char* hdrs[1] = {fbg_device_header};
  const char* names[1] = {"fbg_device.cuh"};
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "fbg_jit.cu", 1, hdrs, names) != NVRTC_SUCCESS) return false;
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


// ---------------------------------------------------- many at once --
// A pool of worker threads compiles many sources (the batch's specialised
// kernels), each cached per source like jit_compile.

namespace {


// one NVRTC compilation to a cubin
bool nvrtc_cubin(const std::string& src, std::string* cubin, std::string* log) {
  const char* hdrs[1] = {fbg_device_header};
  const char* names[1] = {"fbg_device.cuh"};
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "fbg_jit.cu", 1, hdrs, names) != NVRTC_SUCCESS) return false;
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-lineinfo"};
  nvrtcResult e = nvrtcCompileProgram(prog, 3, opts);
  size_t logn = 0;
  nvrtcGetProgramLogSize(prog, &logn);
  if (log && logn > 1) {
    log->resize(logn);
    nvrtcGetProgramLog(prog, &(*log)[0]);
  }
  bool ok = e == NVRTC_SUCCESS;
  if (ok) {
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin->assign(n, '\0');
    nvrtcGetCUBIN(prog, &(*cubin)[0]);
  }
  nvrtcDestroyProgram(&prog);
  return ok;
}

// the sources not yet cached are compiled by the pool; sources still
// compiling at the deadline are reported as not ok (their compiles finish in
// the background)
std::mutex g_cubin_mu;
std::unordered_map<std::string, std::string> g_cubin_cache;   // source -> cubin

std::vector<bool> compile_many(const std::vector<std::string>& bodies, std::vector<std::string>* cubins,
                               double deadline_s, std::string* log) {
  std::mutex& cmu = g_cubin_mu;
  std::unordered_map<std::string, std::string>& cache = g_cubin_cache;
  const size_t n = bodies.size();
  cubins->assign(n, std::string());
  std::vector<bool> ok(n, false);
  struct Pool {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::string> src;
    std::vector<std::string> out;
    std::vector<int> state;   // 0 queued, 1 running, 2 done ok, 3 failed
    size_t next = 0, finished = 0;
    std::string log;
  };
  auto pool = std::make_shared<Pool>();
  for (size_t i = 0; i < n; i++) {
    std::string src = "#include \"fbg_device.cuh\"\n" + bodies[i];
    std::lock_guard<std::mutex> lk(cmu);
    auto it = cache.find(src);
    pool->src.push_back(src);
    if (it != cache.end()) {
      pool->out.push_back(it->second);
      pool->state.push_back(2);
      pool->finished++;
    } else {
      pool->out.push_back(std::string());
      pool->state.push_back(0);
    }
  }
  unsigned workers = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 16u));
  for (unsigned w = 0; w < workers; w++) {
    std::thread([pool, n, &cmu, &cache] {
      for (;;) {
        size_t i;
        {
          std::lock_guard<std::mutex> lk(pool->mu);
          while (pool->next < n && pool->state[pool->next] != 0) pool->next++;
          if (pool->next >= n) return;
          i = pool->next++;
          pool->state[i] = 1;
        }
        std::string cubin, lg;
        bool good = nvrtc_cubin(pool->src[i], &cubin, &lg);
        if (good) {
          std::lock_guard<std::mutex> lk(cmu);
          cache.emplace(pool->src[i], cubin);
        }
        std::lock_guard<std::mutex> lk(pool->mu);
        pool->out[i] = std::move(cubin);
        pool->state[i] = good ? 2 : 3;
        if (!good && pool->log.size() < 4096) pool->log += lg;
        pool->finished++;
        pool->cv.notify_all();
      }
    }).detach();
  }
  std::unique_lock<std::mutex> lk(pool->mu);
  pool->cv.wait_for(lk, std::chrono::duration<double>(deadline_s), [&] { return pool->finished >= n; });
  for (size_t i = 0; i < n; i++) {
    if (pool->state[i] == 2) {
      (*cubins)[i] = pool->out[i];
      ok[i] = true;
    }
  }
  if (log) *log = pool->log;
  if (pool->finished < n && log) *log += "\nsome programs were still compiling at the deadline and run interpreted";
  return ok;
}

// load a complete cubin (cached by key) and look up `kernel_name`
JitResult load_cubin(const std::string& key, const std::string& cubin, const char* kernel_name) {
  JitResult r;
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

}  // namespace

std::vector<JitResult> jit_compile_many(const std::vector<std::string>& bodies, const char* kernel_name, int device,
                                        double deadline_s, std::string* log) {
  const size_t n = bodies.size();
  std::vector<JitResult> res(n);
  std::vector<std::string> todo;
  std::vector<size_t> where;
  for (size_t i = 0; i < n; i++) {
    std::string key = std::to_string(device) + ":" + kernel_name + ":#include \"fbg_device.cuh\"\n" + bodies[i];
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      res[i].ok = true;
      res[i].cached = true;
      res[i].kernel = it->second.kern;
    } else {
      todo.push_back(bodies[i]);
      where.push_back(i);
    }
  }
  if (todo.empty()) return res;
  std::vector<std::string> cubins;
  std::vector<bool> ok = compile_many(todo, &cubins, deadline_s, log);
  for (size_t t = 0; t < todo.size(); t++) {
    if (!ok[t]) continue;
    std::string key = std::to_string(device) + ":" + kernel_name + ":#include \"fbg_device.cuh\"\n" + todo[t];
    res[where[t]] = load_cubin(key, cubins[t], kernel_name);
  }
  return res;
}

std::vector<bool> jit_check_many(const std::vector<std::string>& bodies, double deadline_s, std::string* log) {
  std::vector<std::string> cubins;
  return compile_many(bodies, &cubins, deadline_s, log);
}

size_t jit_cache_size() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_cache.size();
}

}  // namespace fbg
