// Inverse instantiation of the fused kernel (own translation unit: builds in parallel).
#include "adjtx_fused.cuh"

namespace adjtx {

const void* fused_inv_ptr() { return reinterpret_cast<const void*>(&fused_kernel<true, 64>); }

}  // namespace adjtx
