// Forward of FP32 blocks (own translation unit): the fused kernel with FP32 staging, for
// inputs that are not int16 residuals (gradients with respect to the input, filtered data).
#include "adjtx_fused.cuh"

namespace adjtx {

const void* fwd_f32_kernel_ptr() { return reinterpret_cast<const void*>(&fused_kernel<false, 64, kModePackedF32>); }

cudaError_t launch_fwd_f32(int grid, const FusedArgs& args, cudaStream_t stream) {
  FusedArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(fwd_f32_kernel_ptr(), dim3(grid), dim3(64), params, fused_dyn_smem(false, kModePackedF32), stream);
}

}  // namespace adjtx
