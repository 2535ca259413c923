// kernels.hpp -- host-side launchers of the device kernels.
#pragma once

#include <cuda_runtime.h>

#include "fbg_device.cuh"
#include "interp_format.h"

namespace fbg {

size_t interp_smem_bytes(unsigned nslots);
cudaError_t launch_interp(int mode, const FbgInterpProg* progs, const FbgWorkItem* items, unsigned long long nitems,
                          unsigned long long* item_ctr, unsigned long long* prog_counts,
                          unsigned long long* unit_counts, const FbgLaunch& P, unsigned nslots, int grid,
                          cudaStream_t stream, const FbgSlotOut* slot_out = nullptr);
cudaError_t launch_scan(const unsigned long long* in, unsigned long long* out, unsigned long long n,
                        unsigned long long* total, cudaStream_t stream);
int interp_blocks_per_sm(int mode, unsigned nslots);
// out[i] = value for i < n
cudaError_t launch_fill_u64(unsigned long long* out, unsigned long long n, unsigned long long value,
                            cudaStream_t stream);

}  // namespace fbg
