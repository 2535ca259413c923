// noalloc.cu -- model counting without any device allocation by the library.
//
// fbg_count (the normal entry point) allocates the compiled program's device
// buffers and its scratch with cudaMalloc on first use.  Some callers cannot
// allow that: code that must stay inside a fixed, pre-reserved memory budget
// (for example a process whose allocator owns all device memory, or a caller
// that has already handed every free byte to a caching allocator), and code
// paths where an allocation could block or fail at a bad moment.  For them,
// fbg_count_noalloc runs the interpreter count kernel with everything it
// needs besides its output -- work counters, the program descriptor, the
// bytecode, its constants and the work queue -- placed in one file-scope
// device array of fixed size, FBG_NOALLOC_SCRATCH_BYTES (128 KiB), which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "emit.hpp"
#include "fbg.h"
#include "kernels.hpp"
#include "program.hpp"

namespace {

constexpr size_t kWords = FBG_NOALLOC_SCRATCH_BYTES / 8;
constexpr int kMaxDevices = 64;
constexpr uint64_t kMaxItems = 1024;

// the shared scratch: [0] item counter, [1] unused, then the descriptor,
// work items, bytecode and constants, each 16-byte aligned
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kWords];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

using namespace fbg;

extern "C" fbg_status fbg_count_noalloc(fbg_program* p, void* stream, uint64_t* dev_out) {
  if (!p || !dev_out) return set_error(FBG_EINVAL, "null argument");
  if (p->n > 63) return set_error(FBG_ETOOBIG, "counts need n <= 63");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(FBG_EINVAL, "device index out of range");
  // one-time set-up per device (with that device current): host code needs
  // the array's device address; the symbol itself is only a host-side stand-in
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      }
    }
    base = g_scratch_addr[dev];
  }
  // host-side compilation into bytecode (host memory only)
  InterpCode code;
  try {
    // the layout, order and prune points of the interpreter's count build
    Layout L = make_layout(p->n, interp_params(p), order_for(p, true));
    LutProgram prog = lower_and_map(*p->g, L);
    if (!p->opt_prune) strip_prune(prog);
    code = emit_bytecode(prog);
  } catch (CompileError& ce) {
    return set_error(FBG_ETOOBIG, ce.msg);
  }
  const uint64_t nunits = code.prog.nunits;
  const uint64_t per = std::max<uint64_t>(1, (nunits + kMaxItems - 1) / kMaxItems);
  std::vector<FbgWorkItem> items;
  for (uint64_t u = 0; u < nunits; u += per) items.push_back(FbgWorkItem{0u, 0u, u, std::min(nunits, u + per)});
  // placement inside the array
  size_t off_desc = 16;
  size_t off_items = align16(off_desc + sizeof(FbgInterpProg));
  size_t off_ins = align16(off_items + items.size() * sizeof(FbgWorkItem));
  size_t off_consts = align16(off_ins + code.ins.size() * 8);
  size_t need = align16(off_consts + code.consts.size() * 8);
  if (need > FBG_NOALLOC_SCRATCH_BYTES)
    return set_error(FBG_ETOOBIG, "program needs " + std::to_string(need) + " bytes of scratch; fbg_count_noalloc holds at most " +
                                      std::to_string((size_t)FBG_NOALLOC_SCRATCH_BYTES));
  char* b = static_cast<char*>(base);
  FbgInterpProg G = code.prog;
  G.ins = reinterpret_cast<const unsigned long long*>(b + off_ins);
  G.consts = reinterpret_cast<const unsigned long long*>(b + off_consts);
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: counters and the output
  // start from zero, everything else is overwritten
  if ((e = cudaMemsetAsync(b, 0, 16, st)) != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(scratch)");
  if ((e = cudaMemsetAsync(dev_out, 0, 8, st)) != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(out)");
  if ((e = cudaMemcpyAsync(b + off_desc, &G, sizeof G, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync(descriptor)");
  if ((e = cudaMemcpyAsync(b + off_items, items.data(), items.size() * sizeof(FbgWorkItem), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync(items)");
  if (!code.ins.empty() &&
      (e = cudaMemcpyAsync(b + off_ins, code.ins.data(), code.ins.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync(bytecode)");
  if (!code.consts.empty() && (e = cudaMemcpyAsync(b + off_consts, code.consts.data(), code.consts.size() * 8,
                                                   cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_error(e, "cudaMemcpyAsync(constants)");
  int per_sm = interp_blocks_per_sm(0, code.nslots);
  if (per_sm <= 0) return set_error(FBG_ETOOBIG, "interpreter program does not fit in shared memory");
  int grid = (int)std::min<uint64_t>(items.size(), (uint64_t)device_sms() * (uint64_t)per_sm);
  FbgLaunch P{};
  P.unit_begin = 0;
  P.unit_end = nunits;
  e = launch_interp(0, reinterpret_cast<const FbgInterpProg*>(b + off_desc),
                    reinterpret_cast<const FbgWorkItem*>(b + off_items), items.size(),
                    reinterpret_cast<unsigned long long*>(b), reinterpret_cast<unsigned long long*>(dev_out), nullptr,
                    P, code.nslots, grid, st);
  if (e != cudaSuccess) return cuda_error(e, "interpreter launch");
  // pageable host sources: wait until the copies have been consumed before
  // the host buffers above go out of scope
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  return FBG_OK;
}
