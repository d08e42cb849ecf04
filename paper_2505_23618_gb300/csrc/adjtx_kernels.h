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
  // Per-block auxiliary offsets / 4, parallel to tile_blk: the side offsets of the Multiple
  // forward, or the frame offsets (y * frame_stride + x) of blocks inside a frame
  const uint32_t* tile_aux;
  float* side;                // Multiple forward: side buffer
  int64_t frame_stride;       // frame modes: samples per frame row
};

// Kernel modes (template argument of the fused kernel).
enum { kModePacked = 0, kModeMulti = 1, kModeFrame = 2, kModeFrameI16 = 3, kModePackedF32 = 4 };

// Dynamic shared memory of a fused-kernel instantiation: int16 input (forward from packed
// blocks, frames, and the Multiple forward) has its own staging buffer beside one FP32 tile
// buffer; FP32 input is staged in place into two tile buffers.
ADJ_HD bool fused_i16_input(bool inverse, int mode) { return !inverse && mode != kModePackedF32; }
ADJ_HD int fused_dyn_smem(bool inverse, int mode) {
  return fused_i16_input(inverse, mode) ? kSmemBytesI16 : kSmemBytes;
}

// Plain (unfused) form: the blocks of one size class, each with its own transforms.
struct PlainBlock {
  uint32_t off16;
  uint16_t tf_h, tf_v;
};
struct PlainClass {
  int w, h, n_blocks;
  const PlainBlock* blocks;  // device
};
cudaError_t launch_plain(bool inverse, const PlainClass* classes, int n_classes, const TfDev* tfs, const float* P,
                         const void* in, float* out, cudaStream_t stream);

// Backward (parameter and input gradients).
constexpr int kBwdThreads = 128;
struct BwdArgs {
  const TileDev* tiles;
  const uint32_t* tile_blk;
  const TfDev* tfs;
  const float* params;
  const void* x;        // int16 or FP32 input of the forward
  const float* gy;      // dL/dY
  float* gx;            // dL/dX (may be null)
  float* partial;       // [grid][P] per-CTA sums
  const int* m_off;     // per transform: offset of its accumulator in a row of `partial`
  int n_tiles;
  int P;
};
int bwd_smem_bytes();
const void* bwd_kernel_ptr(bool i16);
cudaError_t launch_bwd(bool i16, int grid, const BwdArgs& args, double* M, const TfDev* tfs, int n_tfs,
                       const int* m_off, const int* g_off, const int* kq, float* gparams, cudaStream_t stream);

const void* fused_kernel_ptr(bool inverse, int threads);
const void* multi_kernel_ptr();
cudaError_t launch_multi(int grid, const FusedArgs& args, cudaStream_t stream);
// frame modes: forward reads int16 blocks from a frame; inverse writes FP32 or rounded int16
const void* frame_kernel_ptr(bool inverse, bool i16);
cudaError_t launch_frame(bool inverse, bool i16, int grid, const FusedArgs& args, cudaStream_t stream);
// Forward over packed FP32 input (kModePackedF32), for inputs that are not int16 residuals.
const void* fwd_f32_kernel_ptr();
cudaError_t launch_fwd_f32(int grid, const FusedArgs& args, cudaStream_t stream);
const void* fused_fwd_ptr();
const void* fused_inv_ptr();
void set_last_error(const char* msg);
cudaError_t launch_fused(bool inverse, int threads, int grid, const FusedArgs& args, cudaStream_t stream);

}  // namespace adjtx
