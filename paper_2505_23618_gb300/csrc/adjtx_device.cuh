// Device building blocks of the adjusted transforms: line accessors, the band
// pre-adjustment, the top-left post-adjustment and the 1-D line transform.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_layout.h"
#include "cores_gen.cuh"

namespace adjtx {

// ---------------------------------------------------------------------------------
// Element types.  T = float: one line per thread.  T = float2: two lines per thread,
// element j of line 0 in .x and of line 1 in .y, processed by the packed FP32x2
// instructions (one instruction per operation for both lines).  Runtime coefficients (cos,
// sin of a rotation, entries of Q) are shared by both lines: they are loaded once as scalars
// and broadcast to both halves of the FP32x2 operand, which costs no extra instruction.
// ---------------------------------------------------------------------------------
// log2 of a power of two at run time (one instruction instead of a loop).
__device__ __forceinline__ int lg2(int x) { return 31 - __clz(x); }

__device__ __forceinline__ float vmulv(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vmulv(float2 a, float2 b) { return __fmul2_rn(a, b); }

// ---------------------------------------------------------------------------------
// Fast cores (Section 2.1).  Cores 0..3 are DCT-2, DCT-3, DST-2, DST-3; the inverse of
// each is its transpose, which is the core with index c ^ 1.
// ---------------------------------------------------------------------------------
// PAIR64: 64-point lines run the packed-pair form of the cores (two 32-point cores in one
// FP32x2 pass and a prefix chain: 340 instead of 600 instructions).  It needs a few more live
// registers than the scalar flow graph, which the 168-register kernels have and the
// 128-register int16-input kernels do not, so those keep the scalar graph.
template <int N, bool PAIR64 = false, class T>
__device__ __forceinline__ void core_apply(int core, T (&v)[N]) {
  if constexpr (N == 64 && PAIR64) {
    switch (core) {
      case 0: CorePair64<0>::apply(v); break;
      case 1: CorePair64<1>::apply(v); break;
      case 2: CorePair64<2>::apply(v); break;
      default: CorePair64<3>::apply(v); break;
    }
  } else {
    switch (core) {
      case 0: Core<N, 0>::apply(v); break;
      case 1: Core<N, 1>::apply(v); break;
      case 2: Core<N, 2>::apply(v); break;
      default: Core<N, 3>::apply(v); break;
    }
  }
}

// ---------------------------------------------------------------------------------
// Band pre-adjustment A: layers of disjoint adjacent-pair Givens rotations.
// Forward: layer 0 first, (x_i, x_{i+1}) -> (c x_i - s x_{i+1}, s x_i + c x_{i+1}).
// Inverse (A^T): last layer first, each rotation transposed.
// ---------------------------------------------------------------------------------
// Rotation j of layer l comes from the per-layer table (TfDev::csl_off): rotations 2m and
// 2m + 1 of a layer share one 16-byte load.  Lines of packed pairs broadcast each coefficient.
__device__ __forceinline__ float bc(float x, float) { return x; }
__device__ __forceinline__ float2 bc(float x, float2) { return make_float2(x, x); }

// Negation written per component, so that it folds into the FP32x2 FMA consuming it (one
// instruction less per rotation than a product with -1).  The inverse keeps the product form:
// with the folded one its register allocation changed and it ran about 1 % slower.
__device__ __forceinline__ float rneg(float a) { return -a; }
__device__ __forceinline__ float2 rneg(float2 a) { return make_float2(-a.x, -a.y); }

template <bool INV, class T>
__device__ __forceinline__ void rotate(T& x, T& y, T c, T s) {
  const T a = x, b = y;
  if (!INV) {
    x = vfma(c, a, rneg(vmulv(s, b)));
    y = vfma(c, b, vmulv(s, a));
  } else {
    x = vfma(c, a, vmulv(s, b));
    y = vfma(c, b, vneg(vmulv(s, a)));
  }
}

template <int N, int PAR, bool INV, class T>
__device__ __forceinline__ void rot_layer(T (&v)[N], const float4* __restrict__ cs) {
  constexpr int R = (N - PAR) / 2;  // rotations of the layer
#pragma unroll
  for (int m = 0; m < (R + 1) / 2; ++m) {
    const float4 t = __ldg(cs + m);
    const T z{};
    rotate<INV>(v[4 * m + PAR], v[4 * m + PAR + 1], bc(t.x, z), bc(t.y, z));
    if (2 * m + 1 < R) rotate<INV>(v[4 * m + PAR + 2], v[4 * m + PAR + 3], bc(t.z, z), bc(t.w, z));
  }
}

__device__ __forceinline__ int layer_parity(const TfDev& tf, int l) {
  return l < 32 ? (tf.par_lo >> l) & 1 : (tf.par_hi >> (l - 32)) & 1;
}

template <int N, bool INV, class T>
__device__ __forceinline__ void band(T (&v)[N], const TfDev& tf, const float* __restrict__ P) {
  const float4* cs = reinterpret_cast<const float4*>(P) + tf.csl_off;
  if (!INV) {
    for (int l = 0; l < tf.n_layers; ++l) {
      if (layer_parity(tf, l) == 0) {
        rot_layer<N, 0, false>(v, cs + l * (N / 4));
      } else {
        rot_layer<N, 1, false>(v, cs + l * (N / 4));
      }
    }
  } else {
    for (int l = tf.n_layers - 1; l >= 0; --l) {
      if (layer_parity(tf, l) == 0) {
        rot_layer<N, 0, true>(v, cs + l * (N / 4));
      } else {
        rot_layer<N, 1, true>(v, cs + l * (N / 4));
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Post-adjustment C = diag(Q, I): the padded KT x KT block Qp = diag(Q, I_{KT-K}) (row
// major) acts on the first KT outputs.  Forward: y_i = sum_j Qp[i][j] u_j, written out
// directly at runtime index i (several rows per step, independent accumulators).
// Inverse (C^T): u_j = sum_i Qp[i][j] y_i with y_i read back from the source line.
// Four consecutive entries of a Q row load as one float4.
// ---------------------------------------------------------------------------------
// Rows of Qp handled per step: enough independent accumulators for ILP while the Q
// loads the compiler hoists out of the unrolled dot product still fit in registers.
template <int KT, class T>
struct PostRows {
  static constexpr int R = sizeof(T) == 8 ? (KT >= 32 ? 1 : 2) : (KT >= 64 ? 1 : (KT >= 32 ? 2 : 4));
};

// Qp[i][4g .. 4g+3] as element-type coefficients
__device__ __forceinline__ void q_quad(const float* P, const TfDev& tf, int i, int g, float (&q)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(P + tf.q_off + i * tf.kt) + g);
  q[0] = t.x; q[1] = t.y; q[2] = t.z; q[3] = t.w;
}


// One row of the padded Q in registers: row i as KT/4 float4 (for one line or a packed pair).
template <int KT, class T>
struct QRow {
  static constexpr int NQ = KT / 4;
  float4 q[NQ];
  __device__ __forceinline__ void load(const float* __restrict__ P, const TfDev& tf, int i) {
    const float4* base = reinterpret_cast<const float4*>(P + tf.q_off + i * tf.kt);
#pragma unroll
    for (int g = 0; g < NQ; ++g) q[g] = __ldg(base + g);
  }
};
__device__ __forceinline__ float2 bcast(float q) { return make_float2(q, q); }

// Forward row: y_i = sum_j Q[i][j] v_j.  One line per thread: packed FP32x2 along the inputs,
// {acc_even, acc_odd} += {Q[i][j], Q[i][j+1]} * {v_j, v_{j+1}}, halves added at the end.
// Packed line pairs: one FP32x2 FMA per entry with four partial sums.
template <int KT, int N>
__device__ __forceinline__ float post_row(const QRow<KT, float>& r, const float (&v)[N]) {
  float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int g = 0; g < KT / 4; ++g) {
    acc0 = __ffma2_rn(make_float2(r.q[g].x, r.q[g].y), make_float2(v[4 * g], v[4 * g + 1]), acc0);
    acc1 = __ffma2_rn(make_float2(r.q[g].z, r.q[g].w), make_float2(v[4 * g + 2], v[4 * g + 3]), acc1);
  }
  const float2 t = __fadd2_rn(acc0, acc1);
  return t.x + t.y;
}
template <int KT, int N>
__device__ __forceinline__ float2 post_row(const QRow<KT, float2>& r, const float2 (&v)[N]) {
  float2 acc[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
#pragma unroll
  for (int g = 0; g < KT / 4; ++g) {
    const float4 a = r.q[g];
    acc[0] = __ffma2_rn(bcast(a.x), v[4 * g], acc[0]);
    acc[1] = __ffma2_rn(bcast(a.y), v[4 * g + 1], acc[1]);
    acc[2] = __ffma2_rn(bcast(a.z), v[4 * g + 2], acc[2]);
    acc[3] = __ffma2_rn(bcast(a.w), v[4 * g + 3], acc[3]);
  }
  return __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
}

// Software pipelined over rows when two rows fit in registers beside the line (at most 8
// float4 each for one line, 4 for a packed pair, whose data take twice the registers): row
// i + 1's Q loads are in flight while row i is summed.
template <int KT, class T>
constexpr bool kPipeQ = QRow<KT, T>::NQ <= (sizeof(T) == 4 ? 8 : 4);

template <int N, int KT, class T, class Dst>
__device__ __forceinline__ void post_fwd_k(const T (&v)[N], const TfDev& tf, const float* __restrict__ P,
                                           const Dst& dst) {
#pragma unroll
  for (int i = KT; i < N; ++i) dst.put(i, v[i]);
  if constexpr (kPipeQ<KT, T>) {
    QRow<KT, T> qa, qb;
    qa.load(P, tf, 0);
#pragma unroll 1
    for (int i = 0; i < KT; i += 2) {
      qb.load(P, tf, i + 1);
      dst.put_rt(i, post_row<KT>(qa, v));
      if (i + 2 < KT) qa.load(P, tf, i + 2);
      dst.put_rt(i + 1, post_row<KT>(qb, v));
    }
  } else {
#pragma unroll 1
    for (int i = 0; i < KT; ++i) {
      QRow<KT, T> q;
      q.load(P, tf, i);
      dst.put_rt(i, post_row<KT>(q, v));
    }
  }
}

// Inverse: u_j = sum_i Q[i][j] y_i, y_i read back from the source line.  One line per thread:
// pairs {u_j, u_{j+1}} in packed FP32x2 with y_i broadcast; packed line pairs: one FP32x2 FMA
// per entry.  Pipelined over rows like the forward.
template <int KT, class Src>
__device__ __forceinline__ void post_inv_row(const QRow<KT, float>& r, const Src& src, int i, float2 (&u)[KT / 2]) {
  const float t = src.get_rt(i);
  const float2 y = make_float2(t, t);
#pragma unroll
  for (int g = 0; g < KT / 4; ++g) {
    u[2 * g] = __ffma2_rn(make_float2(r.q[g].x, r.q[g].y), y, u[2 * g]);
    u[2 * g + 1] = __ffma2_rn(make_float2(r.q[g].z, r.q[g].w), y, u[2 * g + 1]);
  }
}
template <int KT, class Src>
__device__ __forceinline__ void post_inv_row(const QRow<KT, float2>& r, const Src& src, int i, float2 (&u)[KT]) {
  const float2 y = src.get_rt(i);
#pragma unroll
  for (int g = 0; g < KT / 4; ++g) {
    const float4 a = r.q[g];
    u[4 * g] = __ffma2_rn(bcast(a.x), y, u[4 * g]);
    u[4 * g + 1] = __ffma2_rn(bcast(a.y), y, u[4 * g + 1]);
    u[4 * g + 2] = __ffma2_rn(bcast(a.z), y, u[4 * g + 2]);
    u[4 * g + 3] = __ffma2_rn(bcast(a.w), y, u[4 * g + 3]);
  }
}

template <int N, int KT, class T, class Src>
__device__ __forceinline__ void post_inv_k(T (&v)[N], const TfDev& tf, const float* __restrict__ P, const Src& src) {
  constexpr int NU = sizeof(T) == 4 ? KT / 2 : KT;
  float2 u[NU];
#pragma unroll
  for (int m = 0; m < NU; ++m) u[m] = make_float2(0.f, 0.f);
  if constexpr (kPipeQ<KT, T>) {
    QRow<KT, T> qa, qb;
    qa.load(P, tf, 0);
#pragma unroll 1
    for (int i = 0; i < KT; i += 2) {
      qb.load(P, tf, i + 1);
      post_inv_row<KT>(qa, src, i, u);
      if (i + 2 < KT) qa.load(P, tf, i + 2);
      post_inv_row<KT>(qb, src, i + 1, u);
    }
  } else {
#pragma unroll 1
    for (int i = 0; i < KT; ++i) {
      QRow<KT, T> q;
      q.load(P, tf, i);
      post_inv_row<KT>(q, src, i, u);
    }
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int m = 0; m < KT / 2; ++m) {
      v[2 * m] = u[m].x;
      v[2 * m + 1] = u[m].y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KT; ++j) v[j] = u[j];
  }
}

// Post blocks that run over the whole tile (post_rows_tile / post_cols_tile in adjtx_fused.cuh)
// instead of per line; their per-line form is then not compiled into the fused kernels.  The
// inverse's with KT = n / 2 on 16- to 64-sample lines, before the line pass:
__host__ __device__ constexpr bool post_inv_tiled(int kt, int n) {
  return (n == 16 && kt == 8) || (n == 32 && kt == 16) || (n == 64 && kt == 32);
}

// The forward's only for 64-sample lines with KT = 32 (rows after the row pass, columns after the
// column pass has written its outputs back into the tile; over Qp^T, TfDev::qt_off): for shorter
// lines the per-line form measured faster in the 128-register forward kernels.
__host__ __device__ constexpr bool post_fwd_tiled(int kt, int n) { return n == 64 && kt == 32; }

template <int N, bool TILED = false, class T, class Dst>
__device__ __forceinline__ void post_fwd(const T (&v)[N], const TfDev& tf, const float* __restrict__ P,
                                         const Dst& dst) {
  switch (tf.kt) {
    case 4: post_fwd_k<N, 4>(v, tf, P, dst); break;
    case 8: if constexpr (N >= 8) { post_fwd_k<N, 8>(v, tf, P, dst); } break;
    case 16: if constexpr (N >= 16) { post_fwd_k<N, 16>(v, tf, P, dst); } break;
    case 32: if constexpr (N >= 32 && !(TILED && post_fwd_tiled(32, N))) { post_fwd_k<N, 32>(v, tf, P, dst); } break;
    default: if constexpr (N >= 64) { post_fwd_k<N, 64>(v, tf, P, dst); } break;
  }
}

// TILED: leave out the (N, KT) pairs that post_inv_tiled hands to the tile-wide form.
template <int N, bool TILED = false, class T, class Src>
__device__ __forceinline__ void post_inv(T (&v)[N], const TfDev& tf, const float* __restrict__ P, const Src& src) {
  switch (tf.kt) {
    case 4: post_inv_k<N, 4>(v, tf, P, src); break;
    case 8: if constexpr (N >= 8 && !(TILED && post_inv_tiled(8, N))) { post_inv_k<N, 8>(v, tf, P, src); } break;
    case 16: if constexpr (N >= 16 && !(TILED && post_inv_tiled(16, N))) { post_inv_k<N, 16>(v, tf, P, src); } break;
    case 32: if constexpr (N >= 32 && !(TILED && post_inv_tiled(32, N))) { post_inv_k<N, 32>(v, tf, P, src); } break;
    default: if constexpr (N >= 64) { post_inv_k<N, 64>(v, tf, P, src); } break;
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
  // the column written back in place (forward columns whose post block runs over the tile)
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) const_cast<float*>(p[(i >> SH) & MK])[i * W] = v[i];
  }
  __device__ __forceinline__ void put(int i, float x) const { const_cast<float*>(p[(i >> SH) & MK])[i * W] = x; }
  __device__ __forceinline__ void put_rt(int i, float x) const {
    const_cast<float*>(blk)[i * W + ((((c >> 2) ^ ((i >> SH) & MK))) << 2) + (c & 3)] = x;
  }
};

// Columns c and c + 1 (c even) of a W wide block in a swizzled tile buffer, as one line of
// float2 elements: both sit in the same 16-byte chunk of every row, so each element pair is
// one 8-byte shared load.
template <int W>
struct ColSw2 {
  static constexpr int SH = sw_shift(W), MK = sw_mask(W), NK = MK + 1;
  const float* p[NK];
  const float* blk;
  int c;
  __device__ __forceinline__ ColSw2(const float* block, int col) : blk(block), c(col) {
#pragma unroll
    for (int k = 0; k < NK; ++k) p[k] = block + ((((col >> 2) ^ k)) << 2) + (col & 3);
  }
  template <int N>
  __device__ __forceinline__ void load(float2 (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = *reinterpret_cast<const float2*>(p[(i >> SH) & MK] + i * W);
  }
  __device__ __forceinline__ float2 get_rt(int i) const {
    return *reinterpret_cast<const float2*>(blk + i * W + ((((c >> 2) ^ ((i >> SH) & MK))) << 2) + (c & 3));
  }
};

// Columns c and c + 1 (c even) of an output block in global memory: 8-byte stores, element i
// at p + i * S.  Every output store is a streaming store (evict first): outputs are written
// once, and keeping them out of L1 leaves it to the transform parameters.
template <int S>
struct DstGCol2 {
  float* p;
  __device__ __forceinline__ void put(int i, float2 x) const { __stcs(reinterpret_cast<float2*>(p + i * S), x); }
  __device__ __forceinline__ void put_rt(int i, float2 x) const { __stcs(reinterpret_cast<float2*>(p + i * S), x); }
  template <int N>
  __device__ __forceinline__ void store(const float2 (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(reinterpret_cast<float2*>(p + i * S), v[i]);
  }
};

// Output columns of a block inside a frame (run-time row stride): FP32, or rounded to the
// nearest integer (ties to even) and saturated to int16.  The pair forms write columns c and
// c + 1 (c even) with one 8-byte (FP32) or 4-byte (int16) store.
__device__ __forceinline__ short sat16(float x) {
  const int v = __float2int_rn(x);
  return (short)(v < -32768 ? -32768 : (v > 32767 ? 32767 : v));
}
struct DstFrame {
  float* p;
  int s;
  __device__ __forceinline__ void put(int i, float x) const { __stcs(p + (size_t)i * s, x); }
  __device__ __forceinline__ void put_rt(int i, float x) const { __stcs(p + (size_t)i * s, x); }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(p + (size_t)i * s, v[i]);
  }
};
struct DstFrame2 {
  float* p;
  int s;
  __device__ __forceinline__ void put(int i, float2 x) const { __stcs(reinterpret_cast<float2*>(p + (size_t)i * s), x); }
  __device__ __forceinline__ void put_rt(int i, float2 x) const { __stcs(reinterpret_cast<float2*>(p + (size_t)i * s), x); }
  template <int N>
  __device__ __forceinline__ void store(const float2 (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(reinterpret_cast<float2*>(p + (size_t)i * s), v[i]);
  }
};
struct DstFrameI16 {
  short* p;
  int s;
  __device__ __forceinline__ void put(int i, float x) const { __stcs(p + (size_t)i * s, sat16(x)); }
  __device__ __forceinline__ void put_rt(int i, float x) const { __stcs(p + (size_t)i * s, sat16(x)); }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(p + (size_t)i * s, sat16(v[i]));
  }
};
struct DstFrameI16x2 {
  short* p;
  int s;
  __device__ __forceinline__ void put(int i, float2 x) const {
    __stcs(reinterpret_cast<short2*>(p + (size_t)i * s), make_short2(sat16(x.x), sat16(x.y)));
  }
  __device__ __forceinline__ void put_rt(int i, float2 x) const { put(i, x); }
  template <int N>
  __device__ __forceinline__ void store(const float2 (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) put(i, v[i]);
  }
};

// A column of an output block in global memory (element i at p[i * S]).
template <int S>
struct DstGCol {
  float* p;
  __device__ __forceinline__ void put(int i, float x) const { __stcs(p + i * S, x); }
  __device__ __forceinline__ void put_rt(int i, float x) const { __stcs(p + i * S, x); }
  template <int N>
  __device__ __forceinline__ void store(const float (&v)[N]) const {
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(p + i * S, v[i]);
  }
};

// ---------------------------------------------------------------------------------
// One line of a pass.  Forward: A (band), B (core), C (post).  Inverse: C^T, B^T, A^T.
// ---------------------------------------------------------------------------------
// TILED (forward passes of the fused kernels): a post block that post_fwd_tiled selects is left
// out here and applied over the whole tile afterwards (the line's core outputs are stored).
template <int N, bool INV, bool I16, class T = float, bool TILED = false, class Src, class Dst>
__device__ __forceinline__ void line_transform(const TfDev& tf, const float* __restrict__ P,
                                               const Src& src, const Dst& dst) {
  T v[N];
  if constexpr (I16) {
    src.template load_i16<N>(v);
  } else {
    src.template load<N>(v);
  }
  if constexpr (!INV) {
    if (tf.kind == KIND_BAND) band<N, false>(v, tf, P);
    if (tf.kind != KIND_DENSE) core_apply<N>(tf.core, v);
    if (tf.kind >= KIND_POST && !(TILED && post_fwd_tiled(tf.kt, N))) {
      post_fwd<N, TILED>(v, tf, P, dst);
    } else {
      dst.template store<N>(v);
    }
  } else {
    if (tf.kind >= KIND_POST && !post_inv_tiled(tf.kt, N)) post_inv<N, true>(v, tf, P, src);
    if (tf.kind != KIND_DENSE) core_apply<N, true>(tf.core ^ 1, v);
    if (tf.kind == KIND_BAND) band<N, true>(v, tf, P);
    dst.template store<N>(v);
  }
}

// Two lines seen as one line of float2 elements (line a in .x, line b in .y).
template <class A>
struct Pair {
  A a, b;
  template <int N>
  __device__ __forceinline__ void load(float2 (&v)[N]) const {
    float x[N], y[N];
    a.template load<N>(x);
    b.template load<N>(y);
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = make_float2(x[i], y[i]);
  }
  template <int N>
  __device__ __forceinline__ void load_i16(float2 (&v)[N]) const {
    float x[N], y[N];
    a.template load_i16<N>(x);
    b.template load_i16<N>(y);
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = make_float2(x[i], y[i]);
  }
  __device__ __forceinline__ float2 get_rt(int i) const { return make_float2(a.get_rt(i), b.get_rt(i)); }
  __device__ __forceinline__ void put(int i, float2 x) const {
    a.put(i, x.x);
    b.put(i, x.y);
  }
  __device__ __forceinline__ void put_rt(int i, float2 x) const {
    a.put_rt(i, x.x);
    b.put_rt(i, x.y);
  }
  template <int N>
  __device__ __forceinline__ void store(const float2 (&v)[N]) const {
    float x[N], y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      x[i] = v[i].x;
      y[i] = v[i].y;
    }
    a.template store<N>(x);
    b.template store<N>(y);
  }
};

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

// Tile claims, made by warp 0 of a CTA for the whole CTA.  A CTA starts on the range of
// its SM and claims tiles from it with one atomicAdd each; the claim for a tile is issued
// one pipeline iteration before its result is read (lane 0 holds it meanwhile), so its
// latency is hidden.  When the range is used up, the warp reads every range's counter at
// once (each lane a few ranges), moves to the range with the most unclaimed tiles and
// claims there.  A failed claim means that range's tiles were all taken by other CTAs, so
// it drops out of later searches: the search ends after at most n_ranges failures.
struct Claimer {
  int range = -1;
  unsigned b0 = 0, b1 = 0;  // tiles [b0, b1) of `range`
  unsigned k = 0;           // lane 0: result of the claim in flight

  __device__ __forceinline__ void set_range(const unsigned* __restrict__ begin, int r) {
    range = r;
    b0 = __ldg(begin + r);
    b1 = __ldg(begin + r + 1);
  }
  // One claim on `range`, waited for (all lanes of warp 0; uniform result).
  __device__ __forceinline__ unsigned claim_now(SchedState* s) {
    unsigned v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(&s->pos[range], 1u);
    return __shfl_sync(0xffffffffu, v, 0);
  }
  // Next tile (all lanes of warp 0), or -1 when every tile has been claimed.  The current
  // range is tried first unless the caller already knows it is used up.
  __device__ __noinline__ int grab(SchedState* s, const unsigned* __restrict__ begin, int n_ranges,
                                  bool try_current = true) {
    const int lane = threadIdx.x & 31;
    if (range < 0) set_range(begin, (int)(sm_id() % (unsigned)n_ranges));
    if (try_current) {
      const unsigned c = claim_now(s);
      if (b0 + c < b1) return (int)(b0 + c);
    }
    for (int guard = 0; guard <= n_ranges + 1; ++guard) {
      int best = -1, best_left = 0;
      for (int r = lane; r < n_ranges; r += 32) {
        const int size = (int)(__ldg(begin + r + 1) - __ldg(begin + r));
        const int left = size - (int)*reinterpret_cast<volatile unsigned*>(&s->pos[r]);
        if (left > best_left) {
          best_left = left;
          best = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int l2 = __shfl_xor_sync(0xffffffffu, best_left, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, best, o);
        if (l2 > best_left || (l2 == best_left && r2 > best)) {
          best_left = l2;
          best = r2;
        }
      }
      if (best < 0) return -1;
      set_range(begin, best);
      const unsigned c = claim_now(s);
      if (b0 + c < b1) return (int)(b0 + c);
    }
    return -1;
  }
  // Lane 0 issues the next claim on the current range; its result is read by resolve().
  __device__ __forceinline__ void issue(SchedState* s) {
    if ((threadIdx.x & 31) == 0) k = atomicAdd(&s->pos[range], 1u);
  }
  // All lanes of warp 0: the tile of the claim issued earlier (searching if it failed).
  __device__ __forceinline__ int resolve(SchedState* s, const unsigned* __restrict__ begin, int n_ranges) {
    const unsigned c = __shfl_sync(0xffffffffu, k, 0);
    if (b0 + c < b1) return (int)(b0 + c);
    return grab(s, begin, n_ranges, false);
  }
};

}  // namespace adjtx
