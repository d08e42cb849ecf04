// Device building blocks of the adjusted transforms: line accessors, the band
// pre-adjustment, the top-left post-adjustment and the 1-D line transform.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_layout.h"
#include "cores_gen.cuh"

namespace adjtx {

// ---------------------------------------------------------------------------------
// Fast cores (Section 2.1).  Cores 0..3 are DCT-2, DCT-3, DST-2, DST-3; the inverse of
// each is its transpose, which is the core with index c ^ 1.
// ---------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void core_apply(int core, float (&v)[N]) {
  switch (core) {
    case 0: Core<N, 0>::apply(v); break;
    case 1: Core<N, 1>::apply(v); break;
    case 2: Core<N, 2>::apply(v); break;
    default: Core<N, 3>::apply(v); break;
  }
}

// ---------------------------------------------------------------------------------
// Band pre-adjustment A: layers of disjoint adjacent-pair Givens rotations.
// Forward: layer 0 first, (x_i, x_{i+1}) -> (c x_i - s x_{i+1}, s x_i + c x_{i+1}).
// Inverse (A^T): last layer first, each rotation transposed.
// ---------------------------------------------------------------------------------
template <int N, int PAR, bool INV>
__device__ __forceinline__ void rot_layer(float (&v)[N], const float2* __restrict__ cs) {
#pragma unroll
  for (int p = 0; p < (N - PAR) / 2; ++p) {
    const int i = 2 * p + PAR;
    const float2 t = __ldg(cs + p);
    const float x = v[i], y = v[i + 1];
    if (!INV) {
      v[i] = t.x * x - t.y * y;
      v[i + 1] = t.y * x + t.x * y;
    } else {
      v[i] = t.x * x + t.y * y;
      v[i + 1] = t.x * y - t.y * x;
    }
  }
}

__device__ __forceinline__ int layer_parity(const TfDev& tf, int l) {
  return l < 32 ? (tf.par_lo >> l) & 1 : (tf.par_hi >> (l - 32)) & 1;
}

template <int N, bool INV>
__device__ __forceinline__ void band(float (&v)[N], const TfDev& tf, const float* __restrict__ P) {
  const float2* cs = reinterpret_cast<const float2*>(P) + tf.cs_off;
  if (!INV) {
    int off = 0;
    for (int l = 0; l < tf.n_layers; ++l) {
      if (layer_parity(tf, l) == 0) {
        rot_layer<N, 0, false>(v, cs + off);
        off += N / 2;
      } else {
        rot_layer<N, 1, false>(v, cs + off);
        off += N / 2 - 1;
      }
    }
  } else {
    int off = tf.n_pairs;
    for (int l = tf.n_layers - 1; l >= 0; --l) {
      if (layer_parity(tf, l) == 0) {
        off -= N / 2;
        rot_layer<N, 0, true>(v, cs + off);
      } else {
        off -= N / 2 - 1;
        rot_layer<N, 1, true>(v, cs + off);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Post-adjustment C = diag(Q, I): the padded KT x KT block Qp = diag(Q, I_{KT-K}) (row
// major) acts on the first KT outputs.  Forward: y_i = sum_j Qp[i][j] u_j, written out
// directly at runtime index i (four rows per step, independent accumulators).
// Inverse (C^T): u_j = sum_i Qp[i][j] y_i with y_i read back from the source line.
// ---------------------------------------------------------------------------------
template <int N, int KT, class Dst>
__device__ __forceinline__ void post_fwd_k(const float (&v)[N], const float* __restrict__ Q,
                                           const Dst& dst) {
#pragma unroll
  for (int i = KT; i < N; ++i) dst.put(i, v[i]);
#pragma unroll 1
  for (int i = 0; i < KT; i += 4) {
    const float4* q = reinterpret_cast<const float4*>(Q + i * KT);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int j = 0; j < KT / 4; ++j) {
      const float4 c0 = __ldg(q + j);
      const float4 c1 = __ldg(q + KT / 4 + j);
      const float4 c2 = __ldg(q + 2 * (KT / 4) + j);
      const float4 c3 = __ldg(q + 3 * (KT / 4) + j);
      const float u0 = v[4 * j], u1 = v[4 * j + 1], u2 = v[4 * j + 2], u3 = v[4 * j + 3];
      a0 = fmaf(c0.x, u0, a0); a0 = fmaf(c0.y, u1, a0); a0 = fmaf(c0.z, u2, a0); a0 = fmaf(c0.w, u3, a0);
      a1 = fmaf(c1.x, u0, a1); a1 = fmaf(c1.y, u1, a1); a1 = fmaf(c1.z, u2, a1); a1 = fmaf(c1.w, u3, a1);
      a2 = fmaf(c2.x, u0, a2); a2 = fmaf(c2.y, u1, a2); a2 = fmaf(c2.z, u2, a2); a2 = fmaf(c2.w, u3, a2);
      a3 = fmaf(c3.x, u0, a3); a3 = fmaf(c3.y, u1, a3); a3 = fmaf(c3.z, u2, a3); a3 = fmaf(c3.w, u3, a3);
    }
    dst.put_rt(i, a0);
    dst.put_rt(i + 1, a1);
    dst.put_rt(i + 2, a2);
    dst.put_rt(i + 3, a3);
  }
}

template <int N, int KT, class Src>
__device__ __forceinline__ void post_inv_k(float (&v)[N], const float* __restrict__ Q, const Src& src) {
#pragma unroll
  for (int j = 0; j < KT; ++j) v[j] = 0.f;
#pragma unroll 1
  for (int i = 0; i < KT; i += 4) {
    const float y0 = src.get_rt(i), y1 = src.get_rt(i + 1), y2 = src.get_rt(i + 2), y3 = src.get_rt(i + 3);
    const float4* q = reinterpret_cast<const float4*>(Q + i * KT);
#pragma unroll
    for (int j = 0; j < KT / 4; ++j) {
      const float4 c0 = __ldg(q + j);
      const float4 c1 = __ldg(q + KT / 4 + j);
      const float4 c2 = __ldg(q + 2 * (KT / 4) + j);
      const float4 c3 = __ldg(q + 3 * (KT / 4) + j);
      v[4 * j] = fmaf(c3.x, y3, fmaf(c2.x, y2, fmaf(c1.x, y1, fmaf(c0.x, y0, v[4 * j]))));
      v[4 * j + 1] = fmaf(c3.y, y3, fmaf(c2.y, y2, fmaf(c1.y, y1, fmaf(c0.y, y0, v[4 * j + 1]))));
      v[4 * j + 2] = fmaf(c3.z, y3, fmaf(c2.z, y2, fmaf(c1.z, y1, fmaf(c0.z, y0, v[4 * j + 2]))));
      v[4 * j + 3] = fmaf(c3.w, y3, fmaf(c2.w, y2, fmaf(c1.w, y1, fmaf(c0.w, y0, v[4 * j + 3]))));
    }
  }
}

template <int N, class Dst>
__device__ __forceinline__ void post_fwd(const float (&v)[N], const TfDev& tf,
                                         const float* __restrict__ P, const Dst& dst) {
  const float* Q = P + tf.q_off;
  switch (tf.kt) {
    case 4: post_fwd_k<N, 4>(v, Q, dst); break;
    case 8: if constexpr (N >= 8) { post_fwd_k<N, 8>(v, Q, dst); } break;
    case 16: if constexpr (N >= 16) { post_fwd_k<N, 16>(v, Q, dst); } break;
    case 32: if constexpr (N >= 32) { post_fwd_k<N, 32>(v, Q, dst); } break;
    default: if constexpr (N >= 64) { post_fwd_k<N, 64>(v, Q, dst); } break;
  }
}

template <int N, class Src>
__device__ __forceinline__ void post_inv(float (&v)[N], const TfDev& tf, const float* __restrict__ P,
                                         const Src& src) {
  const float* Q = P + tf.q_off;
  switch (tf.kt) {
    case 4: post_inv_k<N, 4>(v, Q, src); break;
    case 8: if constexpr (N >= 8) { post_inv_k<N, 8>(v, Q, src); } break;
    case 16: if constexpr (N >= 16) { post_inv_k<N, 16>(v, Q, src); } break;
    case 32: if constexpr (N >= 32) { post_inv_k<N, 32>(v, Q, src); } break;
    default: if constexpr (N >= 64) { post_inv_k<N, 64>(v, Q, src); } break;
  }
}

// ---------------------------------------------------------------------------------
// Line accessors.
// ---------------------------------------------------------------------------------

// A staged int16 row in shared memory (16-B aligned when the row is 16 B or longer).
struct SrcRowI16 {
  const int16_t* p;
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
    if constexpr (N == 4) {
      const int2 r = *reinterpret_cast<const int2*>(p);
      v[0] = (float)(int16_t)(r.x & 0xffff); v[1] = (float)(r.x >> 16);
      v[2] = (float)(int16_t)(r.y & 0xffff); v[3] = (float)(r.y >> 16);
    } else {
#pragma unroll
      for (int q = 0; q < N / 8; ++q) {
        const int4 r = reinterpret_cast<const int4*>(p)[q];
        v[8 * q + 0] = (float)(int16_t)(r.x & 0xffff); v[8 * q + 1] = (float)(r.x >> 16);
        v[8 * q + 2] = (float)(int16_t)(r.y & 0xffff); v[8 * q + 3] = (float)(r.y >> 16);
        v[8 * q + 4] = (float)(int16_t)(r.z & 0xffff); v[8 * q + 5] = (float)(r.z >> 16);
        v[8 * q + 6] = (float)(int16_t)(r.w & 0xffff); v[8 * q + 7] = (float)(r.w >> 16);
      }
    }
  }
  __device__ __forceinline__ float get_rt(int i) const { return (float)p[i]; }
};

// A staged FP32 row in shared memory (16-B aligned).
struct SrcRowF32 {
  const float* p;
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 r = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = r.x; v[4 * q + 1] = r.y; v[4 * q + 2] = r.z; v[4 * q + 3] = r.w;
    }
  }
  __device__ __forceinline__ float get_rt(int i) const { return p[i]; }
};

// A row of the transpose buffer T.
struct DstTRow {
  float* p;
  __device__ __forceinline__ void put(int i, float x) const { p[i] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const { p[i] = x; }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
};

// A column of T (element i at p[i * s]).
struct SrcTCol {
  const float* p;
  int s;
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i * s];
  }
  __device__ __forceinline__ float get_rt(int i) const { return p[i * s]; }
};

// A column of an output block in global memory (element i at p[i * s]).
struct DstGCol {
  float* p;
  int s;
  __device__ __forceinline__ void put(int i, float x) const { p[i * s] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const { p[i * s] = x; }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i * s] = v[i];
  }
};

// ---------------------------------------------------------------------------------
// One line of a pass.  Forward: A (band), B (core), C (post).  Inverse: C^T, B^T, A^T.
// ---------------------------------------------------------------------------------
template <int N, bool INV, class Src, class Dst>
__device__ __forceinline__ void line_transform(const TfDev& tf, const float* __restrict__ P,
                                               const Src& src, const Dst& dst) {
  float v[N];
  src.template load<N>(v);
  if (!INV) {
    if (tf.kind == KIND_BAND) band<N, false>(v, tf, P);
    core_apply<N>(tf.core, v);
    if (tf.kind == KIND_POST) {
      post_fwd<N>(v, tf, P, dst);
    } else {
      dst.template store<N>(v);
    }
  } else {
    if (tf.kind == KIND_POST) post_inv<N>(v, tf, P, src);
    core_apply<N>(tf.core ^ 1, v);
    if (tf.kind == KIND_BAND) band<N, true>(v, tf, P);
    dst.template store<N>(v);
  }
}

// ---------------------------------------------------------------------------------
// Asynchronous 16-B global -> shared copies (staging of the input tile).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace adjtx
