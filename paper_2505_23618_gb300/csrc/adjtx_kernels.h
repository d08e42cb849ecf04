// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_layout.h"

namespace adjtx {

struct FusedArgs {
  const TileDev* tiles;
  const uint32_t* tile_blk;   // block offsets / 16, grouped per tile
  const TfDev* tfs;
  const float* params;
  const void* in;             // int16 (forward) or FP32 (inverse)
  float* out;
  SchedState* sched;          // zero between launches
  const unsigned* range_begin;  // n_ranges + 1 tile indices
  int n_tiles;
  int n_ranges;
};

const void* fused_kernel_ptr(bool inverse, int threads);
void set_last_error(const char* msg);
cudaError_t launch_fused(bool inverse, int threads, int grid, const FusedArgs& args, cudaStream_t stream);

}  // namespace adjtx
