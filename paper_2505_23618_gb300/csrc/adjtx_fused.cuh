// Fused, persistent 2-D adjusted-transform kernels (forward and inverse); the two
// directions are instantiated in adjtx_fused_fwd.cu and adjtx_fused_inv.cu.
//
// One CTA processes one tile at a time: a group of blocks that share
// (w, h, tf_h, tf_v), at most 4096 coefficients.  Per tile:
//   1. stage: 16-B cp.async copies of the blocks' input (int16 forward, FP32 inverse)
//      into a swizzled FP32 tile buffer, each input row inside its own row region;
//   2. row pass: one thread per block row loads its row (16-B shared loads), applies the
//      horizontal 1-D transform (band -> core -> post, or the transposed chain for the
//      inverse) in registers and writes the row back in place (16-B shared stores);
//   3. column pass: one thread per block column reads its column, applies the vertical
//      transform and stores the outputs straight to global memory (a warp covers
//      consecutive columns, so each store instruction is coalesced).
// Each CTA owns two tile buffers: the next tile's copies are in flight while the current
// tile is transformed.  Tiles are sorted by class and cut into per-SM ranges (SchedState),
// so the CTAs resident on an SM execute the same code; the last CTA to finish clears the
// scheduling state, so a launch needs no separate reset.  No CTA ever waits for another.
#include <cuda_runtime.h>
#include <stdint.h>

#pragma once

#include "adjtx_device.cuh"
#include "adjtx_kernels.h"

namespace adjtx {

// Issue the asynchronous copies of one tile's input into a tile buffer (block width W):
// FP32 input (the inverse, and the forward of FP32 blocks) or int16 residuals.
template <int W, bool F32, int THREADS>
__device__ __forceinline__ void stage_tile_w(const TileDev& td, const uint32_t* sOff, const void* in, float* buf) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int h = td.h, nb = td.nblk, lgh = lg2(h);
  if constexpr (F32) {
    // FP32 chunks of 4 samples, W/4 per row, chunk q of row r at slot q ^ f(r).  THREADS is a
    // multiple of the chunks per row, so a thread's chunk column q is fixed; blocks of more than
    // THREADS chunks are walked block by block (one offset load per block), smaller ones with a
    // fixed chunk per thread and a block stride.  (For the int16 forward the plain loop below
    // measured faster.)
    constexpr int LG_CPR = ilog2(W / 4), LG_T = ilog2(THREADS);
    static_assert((THREADS & ((1 << LG_CPR) - 1)) == 0, "THREADS must be a multiple of the chunks per row");
    const float* src = static_cast<const float*>(in);
    const int lg_cpb = LG_CPR + lgh;
    const int q = threadIdx.x & ((1 << LG_CPR) - 1);
    if (lg_cpb > LG_T) {
      for (int b = 0; b < nb; ++b) {
        float* bb = buf + (b << (lgh + ilog2(W)));
        const float* sb = src + (size_t)sOff[b] * 16;
        for (int c = threadIdx.x; c < (1 << lg_cpb); c += THREADS) {
          const int r = c >> LG_CPR;
          cp_async16(bb + r * W + ((q ^ ((r >> SH) & MK)) << 2), sb + c * 4);
        }
      }
    } else {
      const int c = threadIdx.x & ((1 << lg_cpb) - 1), r = c >> LG_CPR;
      const int doff = r * W + ((q ^ ((r >> SH) & MK)) << 2);
      for (int b = threadIdx.x >> lg_cpb; b < nb; b += THREADS >> lg_cpb)
        cp_async16(buf + (b << (lgh + ilog2(W))) + doff, src + (size_t)sOff[b] * 16 + c * 4);
    }
  } else if constexpr (W >= 8) {
    // int16 chunks of 8 samples: W/8 per row, placed at FP32 chunk slot q ^ f(r)
    constexpr int LG_CPR = ilog2(W / 8);
    const int lg_cpb = LG_CPR + lgh, total = nb << lg_cpb;
    const int16_t* src = static_cast<const int16_t*>(in);
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int r = gg >> LG_CPR, q = gg & ((1 << LG_CPR) - 1);
      const size_t off = (size_t)sOff[b] * 16;
      cp_async16(buf + (b << (lgh + ilog2(W))) + r * W + ((q ^ ((r >> SH) & MK)) << 2), src + off + gg * 8);
    }
  } else {
    // W = 4: one int16 row is 8 bytes, copied to the start of its 16-byte row region
    const int total = nb * h;
    const int16_t* src = static_cast<const int16_t*>(in);
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lgh, r = g & (h - 1);
      const size_t off = (size_t)sOff[b] * 16;
      cp_async8(buf + b * 4 * h + r * 4, src + off + r * 4);
    }
  }
}

// int16 staging buffer of the forward (kernels with int16 input).  Line l of a tile (block
// l / h, row l % h) holds its w samples at int16 offset l * w; 16-byte chunk q (8 samples) of
// the line sits at chunk slot q ^ g(l), with g spreading 8 consecutive lines over 8 distinct
// 16-byte bank groups (the FP32 swizzle of a line of w / 2 samples, taken on the line index so
// that it also holds across blocks of 4 rows).  Lines of 4 samples (8 bytes) are dense.
template <int W>
__device__ __forceinline__ int s16_swz(int l) {
  if constexpr (W >= 8) {
    return (l >> sw_shift(W / 2)) & sw_mask(W / 2);
  } else {
    return 0;
  }
}

template <int W, int THREADS>
__device__ __forceinline__ void stage_i16_w(const TileDev& td, const uint32_t* sOff, const int16_t* src,
                                            int16_t* S) {
  const int h = td.h, nb = td.nblk, lgh = lg2(h);
  if constexpr (W >= 8) {
    constexpr int LG_CPR = ilog2(W / 8);
    const int lg_cpb = LG_CPR + lgh, total = nb << lg_cpb;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int l = (b << lgh) + (gg >> LG_CPR), q = gg & ((1 << LG_CPR) - 1);
      cp_async16(S + l * W + ((q ^ s16_swz<W>(l)) << 3), src + (size_t)sOff[b] * 16 + gg * 8);
    }
  } else {
    // 4-wide blocks are 8h contiguous bytes in both places: 16-byte copies of two rows each
    const int lg_cpb = lgh - 1, total = nb << lg_cpb;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      cp_async16(S + (b << (lgh + 2)) + gg * 8, src + (size_t)sOff[b] * 16 + gg * 8);
    }
  }
}

template <int W, int THREADS>
__device__ __forceinline__ void stage_frame_i16_w(const TileDev& td, const uint32_t* sAux, const int16_t* frame,
                                                  int64_t stride, int16_t* S) {
  const int h = td.h, nb = td.nblk, lgh = lg2(h);
  if constexpr (W == 4) {
    const int total = nb << lgh;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lgh, r = g & (h - 1);
      cp_async8(S + g * 4, frame + (size_t)sAux[b] * 4 + (size_t)r * stride);
    }
  } else {
    constexpr int LG_CPR = ilog2(W / 8);
    const int lg_cpb = LG_CPR + lgh, total = nb << lg_cpb;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int r = gg >> LG_CPR, q = gg & ((1 << LG_CPR) - 1), l = (b << lgh) + r;
      const uint32_t a = sAux[b];
      const int16_t* src = frame + (size_t)a * 4 + (size_t)r * stride + q * 8;
      int16_t* dst = S + l * W + ((q ^ s16_swz<W>(l)) << 3);
      if ((a & 1u) == 0) {
        cp_async16(dst, src);
      } else {
        cp_async8(dst, src);
        cp_async8(dst + 4, src + 4);
      }
    }
  }
}

template <bool FRAME, int THREADS>
__device__ __forceinline__ void stage_i16(const TileDev& td, const uint32_t* sIdx, const void* in, int64_t stride,
                                          int16_t* S) {
  const int16_t* src = static_cast<const int16_t*>(in);
#define ADJ_STAGE16(W)                                         \
  if constexpr (FRAME) {                                       \
    stage_frame_i16_w<W, THREADS>(td, sIdx, src, stride, S);   \
  } else {                                                     \
    stage_i16_w<W, THREADS>(td, sIdx, src, S);                 \
  }
  switch (td.w) {
    case 4: ADJ_STAGE16(4) break;
    case 8: ADJ_STAGE16(8) break;
    case 16: ADJ_STAGE16(16) break;
    case 32: ADJ_STAGE16(32) break;
    default: ADJ_STAGE16(64) break;
  }
#undef ADJ_STAGE16
}

// One line of the int16 staging buffer (see stage_i16_w).
template <int W>
struct RowS16 {
  const int16_t* p;  // line start
  int f;             // chunk swizzle of this line
  template <int N>
  __device__ __forceinline__ void load_i16(float (&v)[N]) const {
    if constexpr (N == 4) {
      const int2 r = *reinterpret_cast<const int2*>(p);
      v[0] = (float)(int16_t)(r.x & 0xffff); v[1] = (float)(r.x >> 16);
      v[2] = (float)(int16_t)(r.y & 0xffff); v[3] = (float)(r.y >> 16);
    } else {
#pragma unroll
      for (int q = 0; q < N / 8; ++q) {
        const int4 r = *reinterpret_cast<const int4*>(p + ((q ^ f) << 3));
        v[8 * q + 0] = (float)(int16_t)(r.x & 0xffff); v[8 * q + 1] = (float)(r.x >> 16);
        v[8 * q + 2] = (float)(int16_t)(r.y & 0xffff); v[8 * q + 3] = (float)(r.y >> 16);
        v[8 * q + 4] = (float)(int16_t)(r.z & 0xffff); v[8 * q + 5] = (float)(r.z >> 16);
        v[8 * q + 6] = (float)(int16_t)(r.w & 0xffff); v[8 * q + 7] = (float)(r.w >> 16);
      }
    }
  }
};

// Forward from a frame: block b's row r starts at sample (aux_b * 4 + r * stride) of the int16
// frame (stride a multiple of 8).  Each 8-sample chunk q of a row goes to its chunk slot
// q ^ f(r) as one 16-byte copy when the block starts on an 8-sample boundary, else as two
// 8-byte copies (blocks sit on a 4-sample grid); 4-wide rows are one 8-byte copy.
template <int W, int THREADS>
__device__ __forceinline__ void stage_frame_w(const TileDev& td, const uint32_t* sAux, const int16_t* frame,
                                              int64_t stride, float* buf) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int h = td.h, nb = td.nblk, lgh = lg2(h);
  if constexpr (W == 4) {
    const int total = nb << lgh;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lgh, r = g & (h - 1);
      cp_async8(buf + b * 4 * h + r * 4, frame + (size_t)sAux[b] * 4 + (size_t)r * stride);
    }
  } else {
    constexpr int LG_CPR = ilog2(W / 8);
    const int lg_cpb = LG_CPR + lgh, total = nb << lg_cpb;
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int r = gg >> LG_CPR, q = gg & ((1 << LG_CPR) - 1);
      const uint32_t a = sAux[b];
      const int16_t* src = frame + (size_t)a * 4 + (size_t)r * stride + q * 8;
      float* dst = buf + (b << (lgh + ilog2(W))) + r * W + ((q ^ ((r >> SH) & MK)) << 2);
      if ((a & 1u) == 0) {
        cp_async16(dst, src);
      } else {
        cp_async8(dst, src);
        cp_async8(dst + 2, src + 4);
      }
    }
  }
}

template <int THREADS>
__device__ __forceinline__ void stage_frame(const TileDev& td, const uint32_t* sAux, const void* in, int64_t stride,
                                            float* buf) {
  const int16_t* frame = static_cast<const int16_t*>(in);
  switch (td.w) {
    case 4: stage_frame_w<4, THREADS>(td, sAux, frame, stride, buf); break;
    case 8: stage_frame_w<8, THREADS>(td, sAux, frame, stride, buf); break;
    case 16: stage_frame_w<16, THREADS>(td, sAux, frame, stride, buf); break;
    case 32: stage_frame_w<32, THREADS>(td, sAux, frame, stride, buf); break;
    default: stage_frame_w<64, THREADS>(td, sAux, frame, stride, buf); break;
  }
}

template <bool F32, int THREADS>
__device__ __forceinline__ void stage_tile(const TileDev& td, const uint32_t* sOff, const void* in, float* buf) {
  switch (td.w) {
    case 4: stage_tile_w<4, F32, THREADS>(td, sOff, in, buf); break;
    case 8: stage_tile_w<8, F32, THREADS>(td, sOff, in, buf); break;
    case 16: stage_tile_w<16, F32, THREADS>(td, sOff, in, buf); break;
    case 32: stage_tile_w<32, F32, THREADS>(td, sOff, in, buf); break;
    default: stage_tile_w<64, F32, THREADS>(td, sOff, in, buf); break;
  }
}

// Lines of at most 32 samples are transformed two at a time (lines l and l + half share a
// thread, packed FP32x2 arithmetic); 64-sample lines one per thread.
template <int W, bool INV, int THREADS, bool I16 = !INV>
__device__ __forceinline__ void row_pass(const TfDev& tf, const float* __restrict__ P, float* buf, int nb, int h) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int nlines = nb * h;
  if constexpr (W <= 32) {
    const int half = nlines >> 1;  // nb * h is even (h >= 4)
    for (int l = threadIdx.x; l < half; l += THREADS) {
      const int l2 = l + half;
      Pair<RowSw> row{RowSw{buf + l * W, ((l & (h - 1)) >> SH) & MK},
                      RowSw{buf + l2 * W, ((l2 & (h - 1)) >> SH) & MK}};
      line_transform<W, INV, I16, float2, !INV>(tf, P, row, row);
    }
  } else {
    for (int l = threadIdx.x; l < nlines; l += THREADS) {
      const int r = l & (h - 1);
      RowSw row{buf + l * W, (r >> SH) & MK};
      line_transform<W, INV, I16, float, !INV>(tf, P, row, row);
    }
  }
}

// Forward row pass of kernels with int16 input: lines read from the int16 staging buffer S,
// transformed, and written as FP32 rows into the tile buffer.
template <int W, int THREADS>
__device__ __forceinline__ void row_pass_s16(const TfDev& tf, const float* __restrict__ P, const int16_t* S,
                                             float* buf, int nb, int h) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int nlines = nb * h;
  if constexpr (W <= 32) {
    const int half = nlines >> 1;  // nb * h is even (h >= 4)
    for (int l = threadIdx.x; l < half; l += THREADS) {
      const int l2 = l + half;
      const Pair<RowS16<W>> src{RowS16<W>{S + l * W, s16_swz<W>(l)}, RowS16<W>{S + l2 * W, s16_swz<W>(l2)}};
      const Pair<RowSw> dst{RowSw{buf + l * W, ((l & (h - 1)) >> SH) & MK},
                            RowSw{buf + l2 * W, ((l2 & (h - 1)) >> SH) & MK}};
      line_transform<W, false, true, float2, true>(tf, P, src, dst);
    }
  } else {
    for (int l = threadIdx.x; l < nlines; l += THREADS) {
      const RowS16<W> src{S + l * W, s16_swz<W>(l)};
      const RowSw dst{buf + l * W, ((l & (h - 1)) >> SH) & MK};
      line_transform<W, false, true, float, true>(tf, P, src, dst);
    }
  }
}

// ---------------------------------------------------------------------------------
// Post block over a whole tile (Section 2.2): out_j = sum_i M[i][j] in_i on the first KT values
// of every line, i.e. OUT = IN M for the tile's lines at once, with M = Qp for the inverse (C^T,
// before the line pass) and M = Qp^T for the forward (C, after it).  Each thread computes an
// LG-line x OG-output block with OG/2 FP32x2 accumulators per line, reading its lines' in_i from
// the tile and row i of M (OG consecutive entries, 16-byte loads) once per i, so every entry
// loaded serves LG lines; then all threads write their outputs back in place.
// ---------------------------------------------------------------------------------
// The tile-wide functions are called out of line: only some tiles run them, and keeping their
// code out of the kernel's main loop left the other classes' code and schedule as compact as
// before (measured 1 % on the mixed workload, 4-5 % on plain 32x32 tiles).
template <int W, int KT, int THREADS>
__device__ __noinline__ void post_rows_tile(const float* __restrict__ qtab, float* buf, int nlines, int h) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  constexpr int OG = 8;                                         // outputs per thread
  constexpr int NOG = KT / OG;                                  // output groups
  constexpr int G = THREADS / NOG;                              // line groups
  constexpr int LG = (kTileCoefs / W) / G;                      // lines per thread
  static_assert(NOG * G == THREADS && LG * G == kTileCoefs / W, "post tile mapping");
  const int og = threadIdx.x % NOG, lg = threadIdx.x / NOG;
  float* row[LG];
  int f[LG];
  bool ok[LG];
#pragma unroll
  for (int j = 0; j < LG; ++j) {
    const int l = lg + j * G;  // consecutive lines across the threads of a warp
    ok[j] = l < nlines;
    row[j] = buf + (ok[j] ? l : 0) * W;
    f[j] = ((l & (h - 1)) >> SH) & MK;
  }
  float2 acc[LG][OG / 2];
#pragma unroll
  for (int j = 0; j < LG; ++j)
#pragma unroll
    for (int e = 0; e < OG / 2; ++e) acc[j][e] = make_float2(0.f, 0.f);
  const float4* q = reinterpret_cast<const float4*>(qtab) + og * (OG / 4);
#pragma unroll 4
  for (int i = 0; i < KT; ++i) {
    float4 qi[OG / 4];
#pragma unroll
    for (int g = 0; g < OG / 4; ++g) qi[g] = __ldg(q + i * (KT / 4) + g);
#pragma unroll
    for (int j = 0; j < LG; ++j) {
      const float y = row[j][(((i >> 2) ^ f[j]) << 2) + (i & 3)];
      const float2 yy = make_float2(y, y);
#pragma unroll
      for (int g = 0; g < OG / 4; ++g) {
        acc[j][2 * g] = __ffma2_rn(yy, make_float2(qi[g].x, qi[g].y), acc[j][2 * g]);
        acc[j][2 * g + 1] = __ffma2_rn(yy, make_float2(qi[g].z, qi[g].w), acc[j][2 * g + 1]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < LG; ++j) {
    if (!ok[j]) continue;
#pragma unroll
    for (int g = 0; g < OG / 4; ++g) {
      const int c = og * (OG / 4) + g;  // output chunk
      *reinterpret_cast<float4*>(row[j] + ((c ^ f[j]) << 2)) =
          make_float4(acc[j][2 * g].x, acc[j][2 * g].y, acc[j][2 * g + 1].x, acc[j][2 * g + 1].y);
    }
  }
  __syncthreads();
}

// The same along the columns: out_j = sum_i M[i][j] in_i down each column (rows i < KT of every
// block).  A thread holds 4 adjacent columns (one 16-byte chunk of a row,
// two FP32x2 lanes) x OG outputs for CPT chunks.
template <int H, int KT, int THREADS>
__device__ __noinline__ void post_cols_tile(const float* __restrict__ qtab, float* buf, int nb, int w) {
  constexpr int OG = 8;
  constexpr int NOG = KT / OG;
  constexpr int G = THREADS / NOG;                              // chunk-column groups
  constexpr int CPT = (kTileCoefs / H / 4) / G;                 // chunk columns per thread
  static_assert(NOG * G == THREADS && CPT * G == kTileCoefs / H / 4, "post tile mapping");
  const int sh = sw_shift(w), mk = sw_mask(w), cpr = w >> 2, lgc = lg2(cpr);
  const int og = threadIdx.x % NOG, cg = threadIdx.x / NOG;
  const int nchunks = nb * cpr;
  float* base[CPT];
  int cq[CPT];
  bool ok[CPT];
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    const int x = cg + u * G;
    ok[u] = x < nchunks;
    const int b = ok[u] ? x >> lgc : 0;
    cq[u] = x & (cpr - 1);
    base[u] = buf + b * (w * H);
  }
  float2 acc[CPT][OG][2];
#pragma unroll
  for (int u = 0; u < CPT; ++u)
#pragma unroll
    for (int o = 0; o < OG; ++o) acc[u][o][0] = acc[u][o][1] = make_float2(0.f, 0.f);
  const float4* q = reinterpret_cast<const float4*>(qtab) + og * (OG / 4);
#pragma unroll 4
  for (int i = 0; i < KT; ++i) {
    float qs[OG];
#pragma unroll
    for (int g = 0; g < OG / 4; ++g) {
      const float4 t = __ldg(q + i * (KT / 4) + g);
      qs[4 * g] = t.x; qs[4 * g + 1] = t.y; qs[4 * g + 2] = t.z; qs[4 * g + 3] = t.w;
    }
    const int fi = (i >> sh) & mk;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const float4 y = *reinterpret_cast<const float4*>(base[u] + i * w + ((cq[u] ^ fi) << 2));
      const float2 y0 = make_float2(y.x, y.y), y1 = make_float2(y.z, y.w);
#pragma unroll
      for (int o = 0; o < OG; ++o) {
        acc[u][o][0] = __ffma2_rn(make_float2(qs[o], qs[o]), y0, acc[u][o][0]);
        acc[u][o][1] = __ffma2_rn(make_float2(qs[o], qs[o]), y1, acc[u][o][1]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    if (!ok[u]) continue;
#pragma unroll
    for (int o = 0; o < OG; ++o) {
      const int r = og * OG + o;  // output row
      *reinterpret_cast<float4*>(base[u] + r * w + ((cq[u] ^ ((r >> sh) & mk)) << 2)) =
          make_float4(acc[u][o][0].x, acc[u][o][0].y, acc[u][o][1].x, acc[u][o][1].y);
    }
  }
  __syncthreads();
}

// Copy a transformed tile (swizzled rows) to its packed blocks: 16-byte loads and streaming
// stores, a warp covering consecutive chunks of a block.
template <int THREADS>
__device__ __noinline__ void copy_tile_out(const float* buf, const uint32_t* sOff, float* __restrict__ out,
                                              int nb, int w, int h) {
  const int sh = sw_shift(w), mk = sw_mask(w), lgq = lg2(w >> 2), lgb = lgq + lg2(h);
  const int total = nb << lgb;
  for (int g = threadIdx.x; g < total; g += THREADS) {
    const int b = g >> lgb, rq = g & ((1 << lgb) - 1), r = rq >> lgq, q = rq & ((w >> 2) - 1);
    const float4 v = *reinterpret_cast<const float4*>(buf + b * (w * h) + r * w + ((q ^ ((r >> sh) & mk)) << 2));
    __stcs(reinterpret_cast<float4*>(out + (size_t)sOff[b] * 16 + r * w + q * 4), v);
  }
}

// Output of the column pass: packed blocks (OUT 0, at sOff[b] * 16), or blocks inside a
// frame (at sAux[b] * 4, row stride `stride`) as FP32 (OUT 1) or rounded int16 (OUT 2).
template <int H, int W, bool INV, int THREADS, int OUT>
__device__ __forceinline__ void col_pass(const TfDev& tf, const float* __restrict__ P, float* buf,
                                         const uint32_t* sOff, const uint32_t* sAux, float* __restrict__ out, int nb,
                                         int stride) {
  constexpr int lgw = ilog2(W);
  const int nlines = nb * W;
  // forward 64-sample columns with K = 32: core outputs back into the tile, post block over it
  const bool tiled = !INV && H == 64 && tf.kind >= KIND_POST && post_fwd_tiled(tf.kt, H);
  if constexpr (H <= 32) {
    // adjacent columns (c, c + 1) as one packed pair: 8-byte shared loads and global stores
    const int pairs = nlines >> 1;
    for (int l = threadIdx.x; l < pairs; l += THREADS) {
      const int b = (2 * l) >> lgw, c = (2 * l) & (W - 1);
      const ColSw2<W> src(buf + b * (W * H), c);
      if constexpr (OUT == 0) {
        line_transform<H, INV, false, float2>(tf, P, src, DstGCol2<W>{out + (size_t)sOff[b] * 16 + c});
      } else if constexpr (OUT == 1) {
        line_transform<H, INV, false, float2>(tf, P, src, DstFrame2{out + (size_t)sAux[b] * 4 + c, stride});
      } else {
        short* o16 = reinterpret_cast<short*>(out);
        line_transform<H, INV, false, float2>(tf, P, src, DstFrameI16x2{o16 + (size_t)sAux[b] * 4 + c, stride});
      }
    }
  } else {
    for (int l = threadIdx.x; l < nlines; l += THREADS) {
      const int b = l >> lgw, c = l & (W - 1);
      ColSw<W> src(buf + b * (W * H), c);
      if (!INV && OUT == 0 && tiled) {
        line_transform<H, false, false, float, true>(tf, P, src, src);
      } else if constexpr (OUT == 0) {
        line_transform<H, INV, false>(tf, P, src, DstGCol<W>{out + (size_t)sOff[b] * 16 + c});
      } else if constexpr (OUT == 1) {
        line_transform<H, INV, false>(tf, P, src, DstFrame{out + (size_t)sAux[b] * 4 + c, stride});
      } else {
        short* o16 = reinterpret_cast<short*>(out);
        line_transform<H, INV, false>(tf, P, src, DstFrameI16{o16 + (size_t)sAux[b] * 4 + c, stride});
      }
    }
  }
}

template <int H, bool INV, int THREADS, int OUT>
__device__ __forceinline__ void col_dispatch(const TfDev& tf, const float* __restrict__ P, float* buf,
                                             const uint32_t* sOff, const uint32_t* sAux, float* __restrict__ out,
                                             int nb, int w, int stride) {
  switch (w) {
    case 4: col_pass<H, 4, INV, THREADS, OUT>(tf, P, buf, sOff, sAux, out, nb, stride); break;
    case 8: col_pass<H, 8, INV, THREADS, OUT>(tf, P, buf, sOff, sAux, out, nb, stride); break;
    case 16: col_pass<H, 16, INV, THREADS, OUT>(tf, P, buf, sOff, sAux, out, nb, stride); break;
    case 32: col_pass<H, 32, INV, THREADS, OUT>(tf, P, buf, sOff, sAux, out, nb, stride); break;
    default: col_pass<H, 64, INV, THREADS, OUT>(tf, P, buf, sOff, sAux, out, nb, stride); break;
  }
}

// ---------------------------------------------------------------------------------
// "Multiple" forward (Section 2.3): the 2-D DCT-2 of every block plus the coefficients
// of the four (vertical, horizontal) pairings of DST-7 and DCT-8 post-adjustments that
// differ from it.  Every transform is a DCT-2, optionally followed by C = diag(Q, I) with
// K <= n/2 (the DST-7 adjustment); the DCT-8 one is S C S (Eq. 5).  Side regions of one
// block, in floats from its side offset, each row-major (kh, kv: horizontal and vertical
// K, 0 without an adjustment; a, b = 0 for DST-7, 1 for DCT-8):
//   R_a   rows < kv, columns >= kh of the pairings with vertical a:  kv x (w - kh)
//   L_b   rows >= kv, columns < kh of the pairings with horizontal b: (h - kv) x kh
//   X_ab  rows < kv, columns < kh of pairing (a, b):                 kv x kh
// in the order R_0, R_1, L_0, L_1, X_00, X_01, X_10, X_11.
// ---------------------------------------------------------------------------------
struct SideLayout {
  int w, h, kh, kv;
  __device__ __forceinline__ int r(int a) const { return a * kv * (w - kh); }
  __device__ __forceinline__ int l(int b) const { return 2 * kv * (w - kh) + b * (h - kv) * kh; }
  __device__ __forceinline__ int x(int a, int b) const {
    return 2 * kv * (w - kh) + 2 * (h - kv) * kh + (2 * a + b) * kv * kh;
  }
};

// First k outputs of both adjustments of a DCT-2 line v, from one pass over the padded
// KT x KT Q: with e_i = sum over even j of Q[i][j] v_j and o_i = the sum over odd j, the
// DST-7 adjustment gives e_i + o_i and the DCT-8 one, (S Q S v)_i, gives (-1)^i (e_i - o_i).
// emit(i, dst7_i, dct8_i) is called for i < k.
template <int N, int KT, class Emit>
__device__ __forceinline__ void split_post_k(const float (&v)[N], const TfDev& tf, const float* __restrict__ P,
                                             int k, const Emit& emit) {
  constexpr int R = PostRows<KT, float>::R;
#pragma unroll 1
  for (int i = 0; i < k; i += R) {
    // packed FP32x2 along the inputs: the .x halves sum the even columns, .y the odd ones
    float2 acc[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r][0] = acc[r][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int g = 0; g < KT / 4; ++g) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float q[4];
        q_quad(P, tf, i + r, g, q);
        acc[r][0] = __ffma2_rn(make_float2(q[0], q[1]), make_float2(v[4 * g], v[4 * g + 1]), acc[r][0]);
        acc[r][1] = __ffma2_rn(make_float2(q[2], q[3]), make_float2(v[4 * g + 2], v[4 * g + 3]), acc[r][1]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ii = i + r;
      const float2 t = __fadd2_rn(acc[r][0], acc[r][1]);
      const float e = t.x, o = t.y;
      if (ii < k) emit(ii, e + o, (ii & 1) ? o - e : e - o);
    }
  }
}

// K <= n/2, so the padded size is at most max(4, n/2).
template <int N, class Emit>
__device__ __forceinline__ void split_post(const float (&v)[N], const TfDev& tf, const float* __restrict__ P, int k,
                                           const Emit& emit) {
  switch (tf.kt) {
    case 4: split_post_k<N, 4>(v, tf, P, k, emit); break;
    case 8: if constexpr (N >= 16) { split_post_k<N, 8>(v, tf, P, k, emit); } break;
    case 16: if constexpr (N >= 32) { split_post_k<N, 16>(v, tf, P, k, emit); } break;
    default: if constexpr (N >= 64) { split_post_k<N, 32>(v, tf, P, k, emit); } break;
  }
}

// Column pass over the DCT-2 rows: the 2-D DCT-2 of every column, and for the columns
// >= kh the first kv outputs of both vertical adjustments (regions R_0, R_1).
template <int H, int W, int THREADS>
__device__ __forceinline__ void multi_col_dct(const TfDev& tv, const float* __restrict__ P, const float* buf,
                                              const uint32_t* sOff, const uint32_t* sSide, float* __restrict__ out,
                                              float* __restrict__ side, int nb, int kh, int kv) {
  constexpr int lgw = ilog2(W);
  const int nlines = nb * W, wr = W - kh;
  for (int l = threadIdx.x; l < nlines; l += THREADS) {
    const int b = l >> lgw, c = l & (W - 1);
    float v[H];
    ColSw<W>(buf + b * (W * H), c).template load<H>(v);
    Core<H, 0>::apply(v);
    DstGCol<W>{out + (size_t)sOff[b] * 16 + c}.template store<H>(v);
    if (kv > 0 && c >= kh) {
      float* r0 = side + (size_t)sSide[b] * 4 + (c - kh);
      float* r1 = r0 + kv * wr;
      split_post<H>(v, tv, P, kv, [&](int i, float s7, float c8) {
        __stcs(r0 + i * wr, s7);
        __stcs(r1 + i * wr, c8);
      });
    }
  }
}

// Row step: the first kh outputs of both horizontal adjustments of every DCT-2 row,
// written over the row's columns 0..2kh-1 (DST-7 first), which the column pass above has
// finished reading.
template <int W, int KT, int THREADS>
__device__ __forceinline__ void multi_row_adjust_k(const TfDev& th, const float* __restrict__ P, float* buf, int nb,
                                                   int h, int kh) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int nlines = nb * h;
  for (int l = threadIdx.x; l < nlines; l += THREADS) {
    const RowSw row{buf + l * W, ((l & (h - 1)) >> SH) & MK};
    float v[KT];
    row.template load<KT>(v);
    split_post_k<KT, KT>(v, th, P, kh, [&](int i, float s7, float c8) {
      row.put_rt(i, s7);
      row.put_rt(kh + i, c8);
    });
  }
}

template <int W, int THREADS>
__device__ __forceinline__ void multi_row_adjust(const TfDev& th, const float* __restrict__ P, float* buf, int nb,
                                                 int h, int kh) {
  switch (th.kt) {
    case 4: multi_row_adjust_k<W, 4, THREADS>(th, P, buf, nb, h, kh); break;
    case 8: if constexpr (W >= 16) { multi_row_adjust_k<W, 8, THREADS>(th, P, buf, nb, h, kh); } break;
    case 16: if constexpr (W >= 32) { multi_row_adjust_k<W, 16, THREADS>(th, P, buf, nb, h, kh); } break;
    default: if constexpr (W >= 64) { multi_row_adjust_k<W, 32, THREADS>(th, P, buf, nb, h, kh); } break;
  }
}

// Column pass over the horizontally adjusted columns (2kh per block): vertical DCT-2,
// rows >= kv to L_b, and the first kv outputs of both vertical adjustments to X_0b, X_1b.
template <int H, int W, int THREADS>
__device__ __forceinline__ void multi_col_adj(const TfDev& tv, const float* __restrict__ P, const float* buf,
                                              const uint32_t* sSide, float* __restrict__ side, int nb, int kh,
                                              int kv) {
  const int per = 2 * kh, nlines = nb * per;
  const SideLayout L{W, H, kh, kv};
  for (int l = threadIdx.x; l < nlines; l += THREADS) {
    const int b = l / per, c = l - b * per;
    const int hb = c >= kh ? 1 : 0, j = c - hb * kh;
    float v[H];
    ColSw<W>(buf + b * (W * H), c).template load<H>(v);
    Core<H, 0>::apply(v);
    float* sb = side + (size_t)sSide[b] * 4;
    float* lb = sb + L.l(hb) + j;  // row i >= kv of L_b at lb[(i - kv) * kh]
#pragma unroll
    for (int i = 0; i < H; ++i)
      if (i >= kv) __stcs(lb + (i - kv) * kh, v[i]);
    if (kv > 0) {
      float* x0 = sb + L.x(0, hb) + j;
      float* x1 = sb + L.x(1, hb) + j;
      split_post<H>(v, tv, P, kv, [&](int i, float s7, float c8) {
        __stcs(x0 + i * kh, s7);
        __stcs(x1 + i * kh, c8);
      });
    }
  }
}

template <int H, int THREADS>
__device__ __forceinline__ void multi_after_rows(const TfDev& th, const TfDev& tv, const float* __restrict__ P,
                                                 float* buf, const uint32_t* sOff, const uint32_t* sSide,
                                                 float* __restrict__ out, float* __restrict__ side, int nb, int w) {
  const int kh = th.kind == KIND_POST ? th.k : 0, kv = tv.kind == KIND_POST ? tv.k : 0;
#define ADJ_MULTI_W(W)                                                                    \
  {                                                                                       \
    multi_col_dct<H, W, THREADS>(tv, P, buf, sOff, sSide, out, side, nb, kh, kv);         \
    if (kh > 0) {                                                                         \
      __syncthreads();                                                                    \
      multi_row_adjust<W, THREADS>(th, P, buf, nb, H, kh);                                \
      __syncthreads();                                                                    \
      multi_col_adj<H, W, THREADS>(tv, P, buf, sSide, side, nb, kh, kv);                  \
    }                                                                                     \
  }
  switch (w) {
    case 4: ADJ_MULTI_W(4) break;
    case 8: ADJ_MULTI_W(8) break;
    case 16: ADJ_MULTI_W(16) break;
    case 32: ADJ_MULTI_W(32) break;
    default: ADJ_MULTI_W(64) break;
  }
#undef ADJ_MULTI_W
}

// Resident CTAs per SM that shared memory allows for a kernel with dynamic shared memory
// `dyn` and the static records of the fused kernel (aux: the per-block auxiliary lists of
// the Multiple and frame modes); the register budget follows from it, so spills are never
// traded for occupancy that shared memory forbids.
constexpr int fused_static_smem(bool aux) {
  return 2 * (kMaxTileBlocks + 4) * 4 + (aux ? 2 * (kMaxTileBlocks + 4) * 4 : 16) + 4 * 64 + 2 * 16 + 64;
}
constexpr int fused_ctas_per_sm(bool inverse, int mode) {
  return kSmemPerSm / (fused_dyn_smem(inverse, mode) +
                       fused_static_smem(mode == kModeMulti || mode == kModeFrame || mode == kModeFrameI16) +
                       kSmemReservedPerCta);
}

// Copies a small record (a multiple of 16 bytes) from global to shared memory
// asynchronously, spread over the CTA's threads.
template <int THREADS>
__device__ __forceinline__ void copy_async(void* dst, const void* src, int bytes) {
  for (int i = threadIdx.x * 16; i < bytes; i += THREADS * 16)
    cp_async16(static_cast<unsigned char*>(dst) + i, static_cast<const unsigned char*>(src) + i);
}

template <bool INV, int THREADS, int MODE = kModePacked>
__global__ void __launch_bounds__(THREADS, fused_ctas_per_sm(INV, MODE) * 64 / THREADS) fused_kernel(FusedArgs a) {
  constexpr bool MULTI = MODE == kModeMulti;
  constexpr bool FRAME_IN = !INV && MODE == kModeFrame;   // forward reading blocks from a frame
  constexpr int OUT = !INV || MODE < kModeFrame ? 0 : (MODE == kModeFrame ? 1 : 2);
  constexpr bool AUX = MODE == kModeMulti || MODE == kModeFrame || MODE == kModeFrameI16;
  constexpr bool F32_IN = !fused_i16_input(INV, MODE);  // staged input is FP32 (else int16)
  static_assert(!(INV && MULTI), "the Multiple form is forward only");
  static_assert(!(INV && MODE == kModePackedF32), "FP32 input is the inverse's own");
  static_assert(INV || MODE != kModeFrameI16, "int16 output is for the inverse");
  extern __shared__ __align__(16) unsigned char smem[];
  // Records of this CTA's tiles, by the tile's sequence number k in the CTA, in slot k % 2:
  //   sDesc   descriptor of tile k+1: fetched at step (5) of iteration k-1, valid from (1) of k
  //   sOff    block offsets / 16 of tile k+1: fetched at (2) of k, valid from (4) of k; a
  //           tile's list starts at entry blk_begin & 3 (it is copied from the 16-byte aligned
  //           address below it)
  //   sAux    Multiple / frame modes: side or frame offsets / 4, like sOff
  //   sTf     (horizontal, vertical) transform records of tile k+1, like sOff
  // Tile data: FP32 input is staged in place, tile k in buffer k % 2; int16 input has one tile
  // buffer and one int16 staging buffer S.  Tile k+1 is copied in at step (5) of iteration k,
  // while the column pass of tile k runs.  The claim of tile k+2 is issued at (2) and read at
  // (5) of iteration k, so a CTA holds at most two tiles beyond the one it transforms when the
  // work runs out (each stage of a tile's records is a dependent fetch, hidden behind a pass).
  __shared__ __align__(16) uint32_t sOff[2][kMaxTileBlocks + 4];
  __shared__ __align__(16) uint32_t sAux[AUX ? 2 : 1][AUX ? kMaxTileBlocks + 4 : 4];
  __shared__ __align__(16) TfDev sTf[2][2];
  __shared__ __align__(16) TileDev sDesc[2];
  __shared__ int sIdx[2];
  int16_t* const S = reinterpret_cast<int16_t*>(smem + kBufBytes);  // int16 input only
  const int tid = threadIdx.x;
  Claimer cl;  // used by warp 0 only
  auto list_bytes = [](const TileDev& d) { return (((d.blk_begin & 3) + d.nblk + 3) / 4) * 16; };
  // issue the copies of one tile's input: into buffer `buf` (FP32) or S (int16)
  auto stage = [&](const TileDev& d, int slot, float* buf) {
    if constexpr (F32_IN) {
      stage_tile<true, THREADS>(d, sOff[slot] + (d.blk_begin & 3), a.in, buf);
    } else if constexpr (FRAME_IN) {
      stage_i16<true, THREADS>(d, sAux[slot] + (d.blk_begin & 3), a.in, a.frame_stride, S);
    } else {
      stage_i16<false, THREADS>(d, sOff[slot] + (d.blk_begin & 3), a.in, 0, S);
    }
  };

  // Prologue: warp 0 claims two tiles; fetch the records of tile 0 and the descriptor of tile
  // 1, and stage tile 0.
  if (tid < 32) {
    const int t0 = cl.grab(a.sched, a.range_begin, a.n_ranges);
    const int t1 = t0 >= 0 ? cl.grab(a.sched, a.range_begin, a.n_ranges) : -1;
    if (tid == 0) {
      sIdx[0] = t0;
      sIdx[1] = t1;
    }
  }
  __syncthreads();
  int t = sIdx[0], tn = sIdx[1];
  if (t >= 0) {
    const TileDev d0 = a.tiles[t];
    if (tid == 0) {
      sDesc[0] = d0;
      sTf[0][0] = a.tfs[d0.tf_h];
      sTf[0][1] = a.tfs[d0.tf_v];
      if (tn >= 0) sDesc[1] = a.tiles[tn];
    }
    for (int b = tid; b < d0.nblk; b += THREADS) sOff[0][(d0.blk_begin & 3) + b] = a.tile_blk[d0.blk_begin + b];
    if constexpr (AUX) {
      for (int b = tid; b < d0.nblk; b += THREADS) sAux[0][(d0.blk_begin & 3) + b] = a.tile_aux[d0.blk_begin + b];
    }
    __syncthreads();
    stage(d0, 0, reinterpret_cast<float*>(smem));
    cp_async_commit();
  }

  // Per tile k: (1) wait for the copies issued so far, barrier; (2) fetch the block offsets
  // and transform records of tile k+1 (whose descriptor has arrived); warp 0 issues the claim
  // of tile k+2; (3) row pass; (4) wait, barrier; (5) start copying tile k+1's input; warp 0
  // reads the claim of tile k+2 and fetches its descriptor; column pass.
  for (int k = 0;; ++k) {
    const int cur = F32_IN ? (k & 1) : 0;
    float* buf = reinterpret_cast<float*>(smem + cur * kBufBytes);
    // (1)
    cp_async_wait_all();
    __syncthreads();
    if (k > 0) {
      t = tn;
      tn = sIdx[0];
    }
    if (t < 0) break;
    const TileDev td = sDesc[k & 1];
    // (2)
    if (tn >= 0) {
      const TileDev dn = sDesc[(k + 1) & 1];
      copy_async<THREADS>(sOff[(k + 1) & 1], a.tile_blk + (dn.blk_begin & ~3u), list_bytes(dn));
      if constexpr (AUX) copy_async<THREADS>(sAux[(k + 1) & 1], a.tile_aux + (dn.blk_begin & ~3u), list_bytes(dn));
      copy_async<THREADS>(&sTf[(k + 1) & 1][0], a.tfs + dn.tf_h, sizeof(TfDev));
      copy_async<THREADS>(&sTf[(k + 1) & 1][1], a.tfs + dn.tf_v, sizeof(TfDev));
      if (tid < 32) cl.issue(a.sched);
    }
    cp_async_commit();

    // (3) row pass (horizontal transform, length w): in place (FP32 input) or S -> buffer
    const int w = td.w, h = td.h, nb = td.nblk;
    {
      TfDev tf = sTf[k & 1][0];
      if constexpr (MULTI) tf.kind = KIND_NONE;  // the rows get the plain DCT-2 first
      if constexpr (INV) {
        if (tf.kind >= KIND_POST && post_inv_tiled(tf.kt, w)) {
          if (w == 16) post_rows_tile<16, 8, THREADS>(a.params + tf.q_off, buf, nb * h, h);
          else if (w == 32) post_rows_tile<32, 16, THREADS>(a.params + tf.q_off, buf, nb * h, h);
          else post_rows_tile<64, 32, THREADS>(a.params + tf.q_off, buf, nb * h, h);
        }
      }
      if constexpr (F32_IN) {
        switch (w) {
          case 4: row_pass<4, INV, THREADS, false>(tf, a.params, buf, nb, h); break;
          case 8: row_pass<8, INV, THREADS, false>(tf, a.params, buf, nb, h); break;
          case 16: row_pass<16, INV, THREADS, false>(tf, a.params, buf, nb, h); break;
          case 32: row_pass<32, INV, THREADS, false>(tf, a.params, buf, nb, h); break;
          default: row_pass<64, INV, THREADS, false>(tf, a.params, buf, nb, h); break;
        }
      } else {
        switch (w) {
          case 4: row_pass_s16<4, THREADS>(tf, a.params, S, buf, nb, h); break;
          case 8: row_pass_s16<8, THREADS>(tf, a.params, S, buf, nb, h); break;
          case 16: row_pass_s16<16, THREADS>(tf, a.params, S, buf, nb, h); break;
          case 32: row_pass_s16<32, THREADS>(tf, a.params, S, buf, nb, h); break;
          default: row_pass_s16<64, THREADS>(tf, a.params, S, buf, nb, h); break;
        }
      }
    }
    if constexpr (!INV && !MULTI) {
      const TfDev& th = sTf[k & 1][0];
      if (th.kind >= KIND_POST && post_fwd_tiled(th.kt, w)) {
        __syncthreads();
        post_rows_tile<64, 32, THREADS>(a.params + th.qt_off, buf, nb * h, h);
      }
    }
    // (4)
    cp_async_wait_all();
    __syncthreads();
    // (5)
    if (tn >= 0) {
      stage(sDesc[(k + 1) & 1], (k + 1) & 1, reinterpret_cast<float*>(smem + (cur ^ 1) * kBufBytes));
      if (tid < 32) {
        const int t2 = cl.resolve(a.sched, a.range_begin, a.n_ranges);
        // tile k+2 takes the descriptor slot of tile k, which every thread has read at (1)
        if (tid == 0) {
          sIdx[0] = t2;
          if (t2 >= 0) cp_async16(&sDesc[k & 1], a.tiles + t2);
        }
      }
    } else if (tid == 0) {
      sIdx[0] = -1;
    }
    cp_async_commit();
    // column pass (vertical transform, length h), stores to global memory
    const uint32_t* offs = sOff[k & 1] + (td.blk_begin & 3);
    if constexpr (MULTI) {
      const uint32_t* sides = sAux[k & 1] + (td.blk_begin & 3);
      const TfDev th = sTf[k & 1][0], tv = sTf[k & 1][1];
      switch (h) {
        case 4: multi_after_rows<4, THREADS>(th, tv, a.params, buf, offs, sides, a.out, a.side, nb, w); break;
        case 8: multi_after_rows<8, THREADS>(th, tv, a.params, buf, offs, sides, a.out, a.side, nb, w); break;
        case 16: multi_after_rows<16, THREADS>(th, tv, a.params, buf, offs, sides, a.out, a.side, nb, w); break;
        case 32: multi_after_rows<32, THREADS>(th, tv, a.params, buf, offs, sides, a.out, a.side, nb, w); break;
        default: multi_after_rows<64, THREADS>(th, tv, a.params, buf, offs, sides, a.out, a.side, nb, w); break;
      }
    } else {
      const TfDev tf = sTf[k & 1][1];
      const uint32_t* aux = sAux[AUX ? (k & 1) : 0] + (td.blk_begin & 3);
      const int st = (int)a.frame_stride;
      if constexpr (INV) {
        if (tf.kind >= KIND_POST && post_inv_tiled(tf.kt, h)) {
          if (h == 16) post_cols_tile<16, 8, THREADS>(a.params + tf.q_off, buf, nb, w);
          else if (h == 32) post_cols_tile<32, 16, THREADS>(a.params + tf.q_off, buf, nb, w);
          else post_cols_tile<64, 32, THREADS>(a.params + tf.q_off, buf, nb, w);
        }
      }
      switch (h) {
        case 4: col_dispatch<4, INV, THREADS, OUT>(tf, a.params, buf, offs, aux, a.out, nb, w, st); break;
        case 8: col_dispatch<8, INV, THREADS, OUT>(tf, a.params, buf, offs, aux, a.out, nb, w, st); break;
        case 16: col_dispatch<16, INV, THREADS, OUT>(tf, a.params, buf, offs, aux, a.out, nb, w, st); break;
        case 32: col_dispatch<32, INV, THREADS, OUT>(tf, a.params, buf, offs, aux, a.out, nb, w, st); break;
        default: col_dispatch<64, INV, THREADS, OUT>(tf, a.params, buf, offs, aux, a.out, nb, w, st); break;
      }
      if constexpr (!INV && OUT == 0) {
        if (h == 64 && tf.kind >= KIND_POST && post_fwd_tiled(tf.kt, h)) {
          __syncthreads();
          post_cols_tile<64, 32, THREADS>(a.params + tf.qt_off, buf, nb, w);
          copy_tile_out<THREADS>(buf, offs, a.out, nb, w, h);
        }
      }
    }
  }
  cp_async_wait_all();

  // The last CTA out clears the scheduling state for the next launch on this plan.
  __shared__ int sLast;
  if (tid == 0) {
    __threadfence();
    sLast = atomicAdd(&a.sched->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (sLast) {
    for (int i = tid; i < kMaxRanges; i += THREADS) a.sched->pos[i] = 0u;
    if (tid == 0) a.sched->done = 0u;
    __threadfence();
  }
}

}  // namespace adjtx
