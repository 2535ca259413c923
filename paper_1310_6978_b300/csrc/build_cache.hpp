// build_cache.hpp -- shared host products of a kernel build (cache.cpp).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "emit.hpp"
#include "fbg_internal.hpp"

struct fbg_program;

namespace fbg {

// the host half of a specialised-kernel build (JitBuild without device state)
struct JitHost {
  LutProgram lp;
  std::string src;
  std::vector<long long> ops, uops;
  int unrolled_level = -1;
  int block = 256;
  std::vector<uint8_t> alive;   // empty: every item may hold models (or pruning off)
  std::vector<unsigned> items;  // the live items in natural order (empty with alive)
};

// The live-item list of a cached build on one device, shared by every
// program built from it (freed when the last holder lets go), and the
// kernel of that build on that device (owned by the process-wide JIT cache).
struct JitDevice {
  std::shared_ptr<void> items;   // device array of JitHost::items
  void* kernel = nullptr;        // cudaKernel_t
  int blocks_per_sm = 0;         // occupancy of the kernel at its block size
};
std::shared_ptr<JitDevice> jit_device_get(const std::string& key, int device);
void jit_device_put(const std::string& key, int device, std::shared_ptr<JitDevice> v);

// the host half of an interpreter build
struct InterpHost {
  LutProgram lp;
  InterpCode code;
  uint64_t units_per_item = 1;
  std::shared_ptr<const std::vector<uint32_t>> live;   // null: every unit
};

// key of a build: what ("jit"/"interp"), mode or layout, every option that
// shapes the build, the domain size and the text
std::string build_key(const fbg_program* p, const char* what, int mode);
std::shared_ptr<const JitHost> jit_host_get(const std::string& key);
void jit_host_put(const std::string& key, std::shared_ptr<const JitHost> v);
std::shared_ptr<const InterpHost> interp_host_get(const std::string& key);
void interp_host_put(const std::string& key, std::shared_ptr<const InterpHost> v);
void host_caches_clear();
// hits, misses and entries of the compile, specialised-build and
// interpreter-build caches
void host_cache_stats(uint64_t out[9]);

}  // namespace fbg
