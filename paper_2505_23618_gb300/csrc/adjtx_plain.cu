// Plain (unfused) form of the adjusted transforms: the baseline the fused kernels are
// compared with.  For every block size present there is one launch per step of the 1-D
// chain and per direction -- band, core, post along the rows, then along the columns
// (forward), or the transposed steps in reverse order (inverse) -- and every step reads
// and writes FP32 lines in global memory.  One thread per line; each line looks up its
// own block's transform, so blocks of different types share a launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_device.cuh"
#include "adjtx_kernels.h"

namespace adjtx {

namespace {

// A line in global memory, element i at p[i * s].
struct GLine {
  float* p;
  int s;
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[(size_t)i * s];
  }
  __device__ __forceinline__ float get_rt(int i) const { return p[(size_t)i * s]; }
  __device__ __forceinline__ void put(int i, float x) const { p[(size_t)i * s] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const { p[(size_t)i * s] = x; }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) p[(size_t)i * s] = v[i];
  }
};

struct GLineI16 {
  const int16_t* p;
  int s;
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = (float)p[(size_t)i * s];
  }
};

enum { STEP_PRE = 0, STEP_CORE = 1, STEP_POST = 2 };

// One step of the chain on every line of the blocks of one size class.  FIRST: the step
// reads its lines from `in` (int16 forward, FP32 inverse) and copies the lines it does not
// transform; later steps work in place on `out`.
template <int N, bool INV, int STEP, bool ROW, bool FIRST>
__global__ void __launch_bounds__(256) plain_step(const PlainBlock* __restrict__ blocks, int n_lines, int w, int h,
                                                  const TfDev* __restrict__ tfs, const float* __restrict__ P,
                                                  const void* in, float* out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_lines) return;
  const int per = ROW ? h : w;
  const int b = l / per, i = l - b * per;
  const PlainBlock pb = blocks[b];
  const TfDev tf = tfs[ROW ? pb.tf_h : pb.tf_v];
  const size_t base = (size_t)pb.off16 * 16 + (ROW ? (size_t)i * w : (size_t)i);
  const int s = ROW ? 1 : w;
  GLine dst{out + base, s};
  bool applies;
  if (STEP == STEP_PRE) applies = tf.kind == KIND_BAND;
  else if (STEP == STEP_CORE) applies = tf.kind != KIND_DENSE;
  else applies = tf.kind >= KIND_POST;
  if (!FIRST && !applies) return;
  float v[N];
  if constexpr (FIRST && !INV) {
    GLineI16{static_cast<const int16_t*>(in) + base, s}.template load<N>(v);
  } else if constexpr (FIRST) {
    GLine{const_cast<float*>(static_cast<const float*>(in)) + base, s}.template load<N>(v);
  } else {
    dst.template load<N>(v);
  }
  if (!applies) {
    dst.template store<N>(v);
    return;
  }
  if constexpr (STEP == STEP_PRE) {
    band<N, INV>(v, tf, P);
    dst.template store<N>(v);
  } else if constexpr (STEP == STEP_CORE) {
    core_apply<N>(INV ? (tf.core ^ 1) : tf.core, v);
    dst.template store<N>(v);
  } else if constexpr (!INV) {
    post_fwd<N>(v, tf, P, dst);
  } else {
    const GLine src{FIRST ? const_cast<float*>(static_cast<const float*>(in)) + base : out + base, s};
    post_inv<N>(v, tf, P, src);
    dst.template store<N>(v);
  }
}

template <int N, bool INV, int STEP, bool ROW, bool FIRST>
cudaError_t launch_step(const PlainClass& c, const TfDev* tfs, const float* P, const void* in, float* out,
                        cudaStream_t stream) {
  const int n_lines = c.n_blocks * (ROW ? c.h : c.w);
  const int threads = 256;
  plain_step<N, INV, STEP, ROW, FIRST><<<(n_lines + threads - 1) / threads, threads, 0, stream>>>(
      c.blocks, n_lines, c.w, c.h, tfs, P, in, out);
  return cudaGetLastError();
}

template <int N, bool INV, bool ROW>
cudaError_t launch_chain(const PlainClass& c, const TfDev* tfs, const float* P, const void* in, float* out,
                         cudaStream_t stream) {
  // forward: PRE, CORE, POST; inverse: POST, CORE, PRE.  The row chain starts from `in`.
  constexpr int S0 = INV ? STEP_POST : STEP_PRE, S2 = INV ? STEP_PRE : STEP_POST;
  cudaError_t e = launch_step<N, INV, S0, ROW, ROW>(c, tfs, P, in, out, stream);
  if (e == cudaSuccess) e = launch_step<N, INV, STEP_CORE, ROW, false>(c, tfs, P, in, out, stream);
  if (e == cudaSuccess) e = launch_step<N, INV, S2, ROW, false>(c, tfs, P, in, out, stream);
  return e;
}

template <bool INV, bool ROW>
cudaError_t dispatch_chain(int n, const PlainClass& c, const TfDev* tfs, const float* P, const void* in, float* out,
                           cudaStream_t stream) {
  switch (n) {
    case 4: return launch_chain<4, INV, ROW>(c, tfs, P, in, out, stream);
    case 8: return launch_chain<8, INV, ROW>(c, tfs, P, in, out, stream);
    case 16: return launch_chain<16, INV, ROW>(c, tfs, P, in, out, stream);
    case 32: return launch_chain<32, INV, ROW>(c, tfs, P, in, out, stream);
    default: return launch_chain<64, INV, ROW>(c, tfs, P, in, out, stream);
  }
}

}  // namespace

cudaError_t launch_plain(bool inverse, const PlainClass* classes, int n_classes, const TfDev* tfs, const float* P,
                         const void* in, float* out, cudaStream_t stream) {
  for (int i = 0; i < n_classes; ++i) {
    const PlainClass& c = classes[i];
    if (c.n_blocks == 0) continue;
    cudaError_t e = inverse ? dispatch_chain<true, true>(c.w, c, tfs, P, in, out, stream)
                            : dispatch_chain<false, true>(c.w, c, tfs, P, in, out, stream);
    if (e == cudaSuccess)
      e = inverse ? dispatch_chain<true, false>(c.h, c, tfs, P, in, out, stream)
                  : dispatch_chain<false, false>(c.h, c, tfs, P, in, out, stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace adjtx
