// "Multiple" forward instantiation of the fused kernel (Section 2.3; own translation unit).
#include "adjtx_fused.cuh"

namespace adjtx {

const void* multi_kernel_ptr() { return reinterpret_cast<const void*>(&fused_kernel<false, 64, kModeMulti>); }

cudaError_t launch_multi(int grid, const FusedArgs& args, cudaStream_t stream) {
  FusedArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(multi_kernel_ptr(), dim3(grid), dim3(64), params, fused_dyn_smem(false, kModeMulti), stream);
}

}  // namespace adjtx
