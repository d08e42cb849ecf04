// Frame-mode instantiations of the fused kernel (own translation unit): the forward reads
// int16 blocks from their positions in a residual frame; the inverse writes each block back
// to its position in an FP32 frame or, rounded and saturated, in an int16 frame.
#include "adjtx_fused.cuh"

namespace adjtx {

const void* frame_kernel_ptr(bool inverse, bool i16) {
  if (!inverse) return reinterpret_cast<const void*>(&fused_kernel<false, 64, kModeFrame>);
  return i16 ? reinterpret_cast<const void*>(&fused_kernel<true, 64, kModeFrameI16>)
             : reinterpret_cast<const void*>(&fused_kernel<true, 64, kModeFrame>);
}

cudaError_t launch_frame(bool inverse, bool i16, int grid, const FusedArgs& args, cudaStream_t stream) {
  if (!inverse && i16) return cudaErrorInvalidValue;
  FusedArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(frame_kernel_ptr(inverse, i16), dim3(grid), dim3(64), params, fused_dyn_smem(inverse, inverse && i16 ? kModeFrameI16 : kModeFrame), stream);
}

}  // namespace adjtx
