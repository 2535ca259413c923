// emit.hpp -- code generators for the two evaluation kernels.
#pragma once

#include <string>
#include <vector>

#include "fbg_internal.hpp"
#include "interp_format.h"

namespace fbg {

// CUDA source of the specialised kernel (mode 0: count, 1: truth table);
// the caller prepends fbg_device.cuh.
// ops_per_level (optional) receives the lop3.b32 each thread issues per
// execution of each level after folding; unrolled_level (optional) the loop
// level whose 2^b iterations are emitted as one folded straight-line block
// (one "execution" of that level covers all its iterations), or -1.
// popc_cost: the issue cost of one POPC in vector-ALU slots that sets how
// many full adders the count kernel spends per innermost execution (0: none)
std::string emit_cuda_source(const LutProgram& p, int mode, int block, int minblocks,
                             std::vector<long long>* ops_per_level = nullptr, int* unrolled_level = nullptr,
                             bool counters = true, std::vector<long long>* uniform_ops_per_level = nullptr,
                             int popc_cost = 4);

// Count-mode item pieces: an entry of the item list (FbgLaunch::unit_perm) is
// item | s << 28 | q << 24 (item < 2^24): piece q of 2^s equal ranges of the
// first loop level.  The largest s the kernel of layout L takes (0: items
// are not split -- the first loop level is absent or emitted unrolled).
int top_loop_split_bits(const Layout& L);

struct InterpCode {
  FbgInterpProg prog;                 // device pointers left null
  std::vector<unsigned long long> ins;
  std::vector<unsigned long long> consts;
  unsigned nslots = 1;
};

InterpCode emit_bytecode(const LutProgram& p);

}  // namespace fbg
