// Forward instantiation of the fused kernel (own translation unit: builds in parallel).
#include "adjtx_fused.cuh"

namespace adjtx {

const void* fused_fwd_ptr() { return reinterpret_cast<const void*>(&fused_kernel<false, 64>); }

const void* fused_kernel_ptr(bool inverse, int threads) {
  if (threads != 64) return nullptr;
  return inverse ? fused_inv_ptr() : fused_fwd_ptr();
}

cudaError_t launch_fused(bool inverse, int threads, int grid, const FusedArgs& args, cudaStream_t stream) {
  const void* fn = fused_kernel_ptr(inverse, threads);
  if (!fn) return cudaErrorInvalidValue;
  FusedArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, fused_dyn_smem(inverse, kModePacked), stream);
}

}  // namespace adjtx
