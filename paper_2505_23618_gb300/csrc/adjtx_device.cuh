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
// Rows of Qp handled per step: enough independent accumulators for ILP while the Q
// loads the compiler hoists out of the unrolled dot product still fit in registers.
template <int KT>
struct PostRows {
  static constexpr int R = KT >= 64 ? 1 : (KT >= 32 ? 2 : 4);
};

template <int N, int KT, class Dst>
__device__ __forceinline__ void post_fwd_k(const float (&v)[N], const float* __restrict__ Q,
                                           const Dst& dst) {
  constexpr int R = PostRows<KT>::R;
#pragma unroll
  for (int i = KT; i < N; ++i) dst.put(i, v[i]);
#pragma unroll 1
  for (int i = 0; i < KT; i += R) {
    const float4* q = reinterpret_cast<const float4*>(Q + i * KT);
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.f;
#pragma unroll
    for (int j = 0; j < KT / 4; ++j) {
      const float u0 = v[4 * j], u1 = v[4 * j + 1], u2 = v[4 * j + 2], u3 = v[4 * j + 3];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 c = __ldg(q + r * (KT / 4) + j);
        acc[r] = fmaf(c.x, u0, acc[r]);
        acc[r] = fmaf(c.y, u1, acc[r]);
        acc[r] = fmaf(c.z, u2, acc[r]);
        acc[r] = fmaf(c.w, u3, acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) dst.put_rt(i + r, acc[r]);
  }
}

template <int N, int KT, class Src>
__device__ __forceinline__ void post_inv_k(float (&v)[N], const float* __restrict__ Q, const Src& src) {
  constexpr int R = PostRows<KT>::R;
#pragma unroll
  for (int j = 0; j < KT; ++j) v[j] = 0.f;
#pragma unroll 1
  for (int i = 0; i < KT; i += R) {
    float y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = src.get_rt(i + r);
    const float4* q = reinterpret_cast<const float4*>(Q + i * KT);
#pragma unroll
    for (int j = 0; j < KT / 4; ++j) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float4 c = __ldg(q + r * (KT / 4) + j);
        v[4 * j] = fmaf(c.x, y[r], v[4 * j]);
        v[4 * j + 1] = fmaf(c.y, y[r], v[4 * j + 1]);
        v[4 * j + 2] = fmaf(c.z, y[r], v[4 * j + 2]);
        v[4 * j + 3] = fmaf(c.w, y[r], v[4 * j + 3]);
      }
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

// One row of a swizzled tile buffer, transformed in place by the thread that owns it.
// The staged input of the row (int16 forward, FP32 inverse) sits in the row's own region:
// int16 chunk q (8 samples) and FP32 chunk q (4 samples) are both at chunk slot q ^ f.
struct RowSw {
  float* p;  // row start
  int f;     // swizzle of this row
  __device__ __forceinline__ int at(int i) const { return ((((i >> 2) ^ f)) << 2) + (i & 3); }
  template <int N>
  __device__ __forceinline__ void load_i16(float (&v)[N]) const {
    if constexpr (N == 4) {
      const int2 r = *reinterpret_cast<const int2*>(p);
      v[0] = (float)(int16_t)(r.x & 0xffff); v[1] = (float)(r.x >> 16);
      v[2] = (float)(int16_t)(r.y & 0xffff); v[3] = (float)(r.y >> 16);
    } else {
#pragma unroll
      for (int q = 0; q < N / 8; ++q) {
        const int4 r = *reinterpret_cast<const int4*>(p + ((q ^ f) << 2));
        v[8 * q + 0] = (float)(int16_t)(r.x & 0xffff); v[8 * q + 1] = (float)(r.x >> 16);
        v[8 * q + 2] = (float)(int16_t)(r.y & 0xffff); v[8 * q + 3] = (float)(r.y >> 16);
        v[8 * q + 4] = (float)(int16_t)(r.z & 0xffff); v[8 * q + 5] = (float)(r.z >> 16);
        v[8 * q + 6] = (float)(int16_t)(r.w & 0xffff); v[8 * q + 7] = (float)(r.w >> 16);
      }
    }
  }
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 r = *reinterpret_cast<const float4*>(p + ((q ^ f) << 2));
      v[4 * q] = r.x; v[4 * q + 1] = r.y; v[4 * q + 2] = r.z; v[4 * q + 3] = r.w;
    }
  }
  __device__ __forceinline__ float get_rt(int i) const { return p[at(i)]; }
  __device__ __forceinline__ void put(int i, float x) const { p[at(i)] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const { p[at(i)] = x; }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
      *reinterpret_cast<float4*>(p + ((q ^ f) << 2)) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
};

// Column c of a w = W wide block in a swizzled tile buffer.  Element i sits at
// i*W + (((c >> 2) ^ f(i)) << 2) + (c & 3); f(i) takes at most 8 values, so one base
// pointer per value keeps every access a shared load with an immediate offset.
template <int W>
struct ColSw {
  static constexpr int SH = sw_shift(W), MK = sw_mask(W), NK = MK + 1;
  const float* p[NK];
  const float* blk;
  int c;
  __device__ __forceinline__ ColSw(const float* block, int col) : blk(block), c(col) {
#pragma unroll
    for (int k = 0; k < NK; ++k) p[k] = block + ((((col >> 2) ^ k)) << 2) + (col & 3);
  }
  template <int N>
  __device__ __forceinline__ void load(float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[(i >> SH) & MK][i * W];
  }
  __device__ __forceinline__ float get_rt(int i) const {
    return blk[i * W + ((((c >> 2) ^ ((i >> SH) & MK))) << 2) + (c & 3)];
  }
};

// A column of an output block in global memory (element i at p[i * S]).
template <int S>
struct DstGCol {
  float* p;
  __device__ __forceinline__ void put(int i, float x) const { p[i * S] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const { p[i * S] = x; }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i * S] = v[i];
  }
};

// ---------------------------------------------------------------------------------
// One line of a pass.  Forward: A (band), B (core), C (post).  Inverse: C^T, B^T, A^T.
// ---------------------------------------------------------------------------------
template <int N, bool INV, bool I16, class Src, class Dst>
__device__ __forceinline__ void line_transform(const TfDev& tf, const float* __restrict__ P,
                                               const Src& src, const Dst& dst) {
  float v[N];
  if constexpr (I16) {
    src.template load_i16<N>(v);
  } else {
    src.template load<N>(v);
  }
  if (!INV) {
    if (tf.kind == KIND_BAND) band<N, false>(v, tf, P);
    if (tf.kind != KIND_DENSE) core_apply<N>(tf.core, v);
    if (tf.kind >= KIND_POST) {
      post_fwd<N>(v, tf, P, dst);
    } else {
      dst.template store<N>(v);
    }
  } else {
    if (tf.kind >= KIND_POST) post_inv<N>(v, tf, P, src);
    if (tf.kind != KIND_DENSE) core_apply<N>(tf.core ^ 1, v);
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
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Completes a claim whose atomicAdd on s->pos[range] returned k (issued earlier, so its
// latency overlapped other work): the tile index, or the result of a full search when
// the range turned out to be exhausted.
static __device__ int grab_tile(SchedState* s, const unsigned* __restrict__ begin, int n_ranges, int& range);
__device__ __forceinline__ int claim_resolve(SchedState* s, const unsigned* __restrict__ begin, int n_ranges,
                                             int& range, unsigned k) {
  const unsigned t = __ldg(begin + range) + k;
  if (t < __ldg(begin + range + 1)) return (int)t;
  return grab_tile(s, begin, n_ranges, range);
}

// First range after `from` (cyclically) whose bit is clear in the bitmap snapshot, or -1.
__device__ __forceinline__ int next_open_range(const unsigned* ex, int from, int n_ranges) {
  for (int step = 1; step <= n_ranges; ++step) {
    const int r = (from + step) % n_ranges;
    if (!((ex[r >> 5] >> (r & 31)) & 1u)) return r;
  }
  return -1;
}

// Next tile for this CTA (called by one thread), or -1 when every tile is claimed.
// `range` is the CTA's current range (initially -1: start at the SM's own range).
// Every probe either returns a tile or marks one more range exhausted, so the loop ends
// after at most 2 * n_ranges + 2 probes.
static __device__ __noinline__ int grab_tile(SchedState* s, const unsigned* __restrict__ begin, int n_ranges,
                                       int& range) {
  if (range < 0) range = (int)(sm_id() % (unsigned)n_ranges);
  unsigned ex[kMaxRanges / 32];
  bool have = false;
  for (int probes = 0; probes < 2 * n_ranges + 2; ++probes) {
    const unsigned k = atomicAdd(&s->pos[range], 1u);
    const unsigned t = __ldg(begin + range) + k;
    if (t < __ldg(begin + range + 1)) return (int)t;
    atomicOr(&s->exhausted[range >> 5], 1u << (range & 31));
    if (!have) {
      const volatile unsigned* g = s->exhausted;
      for (int i = 0; i < (n_ranges + 31) / 32; ++i) ex[i] = g[i];
      have = true;
    }
    ex[range >> 5] |= 1u << (range & 31);
    int next = next_open_range(ex, range, n_ranges);
    if (next < 0) {
      // the snapshot says everything is taken: confirm with a fresh one
      const volatile unsigned* g = s->exhausted;
      for (int i = 0; i < (n_ranges + 31) / 32; ++i) ex[i] = g[i];
      next = next_open_range(ex, range, n_ranges);
      if (next < 0) return -1;
    }
    range = next;
  }
  return -1;
}

}  // namespace adjtx
