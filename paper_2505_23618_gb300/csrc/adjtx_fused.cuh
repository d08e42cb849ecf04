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

// Issue the asynchronous copies of one tile's input into a tile buffer.
template <bool INV, int THREADS>
__device__ __forceinline__ void stage_tile(const TileDev& td, const uint32_t* sOff, const void* in, float* buf) {
  const int w = td.w, h = td.h, nb = td.nblk;
  const int sh = sw_shift(w), mk = sw_mask(w);
  if constexpr (INV) {
    // FP32 chunks of 4 samples: w/4 per row
    const int lg_cpr = ilog2(w >> 2), lg_cpb = ilog2((w * h) >> 2);
    const int total = nb << lg_cpb;
    const float* src = static_cast<const float*>(in);
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int r = gg >> lg_cpr, q = gg & ((1 << lg_cpr) - 1);
      const size_t off = (size_t)sOff[b] * 16;
      cp_async16(buf + b * w * h + r * w + ((q ^ ((r >> sh) & mk)) << 2), src + off + gg * 4);
    }
  } else if (w >= 8) {
    // int16 chunks of 8 samples: w/8 per row, placed at FP32 chunk slot q ^ f(r)
    const int lg_cpr = ilog2(w >> 3), lg_cpb = ilog2((w * h) >> 3);
    const int total = nb << lg_cpb;
    const int16_t* src = static_cast<const int16_t*>(in);
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lg_cpb, gg = g & ((1 << lg_cpb) - 1);
      const int r = gg >> lg_cpr, q = gg & ((1 << lg_cpr) - 1);
      const size_t off = (size_t)sOff[b] * 16;
      cp_async16(buf + b * w * h + r * w + ((q ^ ((r >> sh) & mk)) << 2), src + off + gg * 8);
    }
  } else {
    // w = 4: one int16 row is 8 bytes, copied to the start of its 16-byte row region
    const int total = nb * h;
    const int16_t* src = static_cast<const int16_t*>(in);
    const int lgh = ilog2(h);
    for (int g = threadIdx.x; g < total; g += THREADS) {
      const int b = g >> lgh, r = g & (h - 1);
      const size_t off = (size_t)sOff[b] * 16;
      cp_async8(buf + b * 4 * h + r * 4, src + off + r * 4);
    }
  }
}

// Lines of at most 32 samples are transformed two at a time (lines l and l + half share a
// thread, packed FP32x2 arithmetic); 64-sample lines one per thread.
template <int W, bool INV, int THREADS>
__device__ __forceinline__ void row_pass(const TfDev& tf, const float* __restrict__ P, float* buf, int nb, int h) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int nlines = nb * h;
  if constexpr (W <= 32) {
    const int half = nlines >> 1;  // nb * h is even (h >= 4)
    for (int l = threadIdx.x; l < half; l += THREADS) {
      const int l2 = l + half;
      Pair<RowSw> row{RowSw{buf + l * W, ((l & (h - 1)) >> SH) & MK},
                      RowSw{buf + l2 * W, ((l2 & (h - 1)) >> SH) & MK}};
      line_transform<W, INV, !INV, float2>(tf, P, row, row);
    }
  } else {
    for (int l = threadIdx.x; l < nlines; l += THREADS) {
      const int r = l & (h - 1);
      RowSw row{buf + l * W, (r >> SH) & MK};
      line_transform<W, INV, !INV>(tf, P, row, row);
    }
  }
}

template <int H, int W, bool INV, int THREADS>
__device__ __forceinline__ void col_pass(const TfDev& tf, const float* __restrict__ P, const float* buf,
                                         const uint32_t* sOff, float* __restrict__ out, int nb) {
  constexpr int lgw = ilog2(W);
  const int nlines = nb * W;
  if constexpr (H <= 32) {
    const int half = nlines >> 1;
    for (int l = threadIdx.x; l < half; l += THREADS) {
      const int l2 = l + half;
      const int b1 = l >> lgw, c1 = l & (W - 1), b2 = l2 >> lgw, c2 = l2 & (W - 1);
      Pair<ColSw<W>> src{ColSw<W>(buf + b1 * (W * H), c1), ColSw<W>(buf + b2 * (W * H), c2)};
      Pair<DstGCol<W>> dst{DstGCol<W>{out + (size_t)sOff[b1] * 16 + c1}, DstGCol<W>{out + (size_t)sOff[b2] * 16 + c2}};
      line_transform<H, INV, false, float2>(tf, P, src, dst);
    }
  } else {
    for (int l = threadIdx.x; l < nlines; l += THREADS) {
      const int b = l >> lgw, c = l & (W - 1);
      ColSw<W> src(buf + b * (W * H), c);
      DstGCol<W> dst{out + (size_t)sOff[b] * 16 + c};
      line_transform<H, INV, false>(tf, P, src, dst);
    }
  }
}

template <int H, bool INV, int THREADS>
__device__ __forceinline__ void col_dispatch(const TfDev& tf, const float* __restrict__ P, const float* buf,
                                             const uint32_t* sOff, float* __restrict__ out, int nb, int w) {
  switch (w) {
    case 4: col_pass<H, 4, INV, THREADS>(tf, P, buf, sOff, out, nb); break;
    case 8: col_pass<H, 8, INV, THREADS>(tf, P, buf, sOff, out, nb); break;
    case 16: col_pass<H, 16, INV, THREADS>(tf, P, buf, sOff, out, nb); break;
    case 32: col_pass<H, 32, INV, THREADS>(tf, P, buf, sOff, out, nb); break;
    default: col_pass<H, 64, INV, THREADS>(tf, P, buf, sOff, out, nb); break;
  }
}

// Shared memory limits residency to kSmemCtasPerSm CTAs per SM; the register budget
// follows from that, so spills are never traded for occupancy that smem forbids.
constexpr int kSmemCtasPerSm = (227 * 1024) / (kSmemBytes + 3072);

// Copies a small record (a multiple of 16 bytes) from global to shared memory
// asynchronously, spread over the CTA's threads.
template <int THREADS>
__device__ __forceinline__ void copy_async(void* dst, const void* src, int bytes) {
  for (int i = threadIdx.x * 16; i < bytes; i += THREADS * 16)
    cp_async16(static_cast<unsigned char*>(dst) + i, static_cast<const unsigned char*>(src) + i);
}

template <bool INV, int THREADS>
__global__ void __launch_bounds__(THREADS, kSmemCtasPerSm * 64 / THREADS) fused_kernel(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  // block offsets / 16 of the tiles in buf[0], buf[1]; a tile's list starts at entry
  // blk_begin & 3 (it is copied from the 16-byte aligned address below blk_begin)
  __shared__ __align__(16) uint32_t sOff[2][kMaxTileBlocks + 4];
  __shared__ __align__(16) TfDev sTf[2][2];                   // (horizontal, vertical) records
  __shared__ __align__(16) TileDev sDesc[3];                  // descriptors, by tile sequence mod 3
  __shared__ int sIdx[3];
  const int tid = threadIdx.x;
  int range = -1;        // thread 0 only: the range claims come from
  unsigned claim_k = 0;  // thread 0 only: pending claim

  // Prologue: claim three tiles, fetch what the first iteration needs, stage tile 0.
  if (tid == 0) {
    sIdx[0] = grab_tile(a.sched, a.range_begin, a.n_ranges, range);
    sIdx[1] = sIdx[0] >= 0 ? grab_tile(a.sched, a.range_begin, a.n_ranges, range) : -1;
    sIdx[2] = sIdx[1] >= 0 ? grab_tile(a.sched, a.range_begin, a.n_ranges, range) : -1;
  }
  __syncthreads();
  int t = sIdx[0], tn = sIdx[1], tn2 = sIdx[2];
  if (t >= 0) {
    const TileDev d0 = a.tiles[t];
    if (tid == 0) {
      sDesc[0] = d0;
      if (tn >= 0) sDesc[1] = a.tiles[tn];
      sTf[0][0] = a.tfs[d0.tf_h];
      sTf[0][1] = a.tfs[d0.tf_v];
    }
    for (int b = tid; b < d0.nblk; b += THREADS) sOff[0][(d0.blk_begin & 3) + b] = a.tile_blk[d0.blk_begin + b];
    __syncthreads();
    stage_tile<INV, THREADS>(d0, sOff[0] + (d0.blk_begin & 3), a.in, reinterpret_cast<float*>(smem));
    if (tn2 >= 0) copy_async<THREADS>(&sDesc[2], a.tiles + tn2, sizeof(TileDev));
    cp_async_commit();
  }

  // Per tile: (1) wait; (2) async-fetch the next tile's metadata; (3) row pass; (4) wait,
  // barrier; (5) stage the next tile; (6) column pass.  Copies of the next tile overlap
  // the column pass of this one and the row pass of the next.
  for (int k = 0, cur = 0; t >= 0; ++k, cur ^= 1) {
    float* buf = reinterpret_cast<float*>(smem + cur * kBufBytes);
    // (1) this tile's data, the next descriptor and this tile's records have landed
    cp_async_wait_all();
    __syncthreads();
    const TileDev td = sDesc[k % 3];
    // (2) fetch the next tile's block offsets and records; claim one more tile
    if (tn >= 0) {
      const TileDev dn = sDesc[(k + 1) % 3];
      copy_async<THREADS>(sOff[cur ^ 1], a.tile_blk + (dn.blk_begin & ~3u),
                          (((dn.blk_begin & 3) + dn.nblk + 3) / 4) * 16);
      copy_async<THREADS>(&sTf[cur ^ 1][0], a.tfs + dn.tf_h, sizeof(TfDev));
      copy_async<THREADS>(&sTf[cur ^ 1][1], a.tfs + dn.tf_v, sizeof(TfDev));
    }
    cp_async_commit();
    if (tid == 0 && tn2 >= 0) claim_k = atomicAdd(&a.sched->pos[range], 1u);

    // (3) row pass (horizontal transform, length w), in place
    const int w = td.w, h = td.h, nb = td.nblk;
    {
      const TfDev tf = sTf[cur][0];
      switch (w) {
        case 4: row_pass<4, INV, THREADS>(tf, a.params, buf, nb, h); break;
        case 8: row_pass<8, INV, THREADS>(tf, a.params, buf, nb, h); break;
        case 16: row_pass<16, INV, THREADS>(tf, a.params, buf, nb, h); break;
        case 32: row_pass<32, INV, THREADS>(tf, a.params, buf, nb, h); break;
        default: row_pass<64, INV, THREADS>(tf, a.params, buf, nb, h); break;
      }
    }
    // (4) the next tile's offsets have landed; publish the claimed tile index
    cp_async_wait_all();
    if (tid == 0) sIdx[k % 3] = tn2 >= 0 ? claim_resolve(a.sched, a.range_begin, a.n_ranges, range, claim_k) : -1;
    __syncthreads();
    const int tn3 = sIdx[k % 3];
    // (5) stage the next tile into the other buffer; fetch the descriptor after it
    if (tn >= 0) {
      const TileDev dn = sDesc[(k + 1) % 3];
      stage_tile<INV, THREADS>(dn, sOff[cur ^ 1] + (dn.blk_begin & 3), a.in,
                               reinterpret_cast<float*>(smem + (cur ^ 1) * kBufBytes));
    }
    if (tn3 >= 0) copy_async<THREADS>(&sDesc[k % 3], a.tiles + tn3, sizeof(TileDev));
    cp_async_commit();
    // (6) column pass (vertical transform, length h), stores to global memory
    {
      const TfDev tf = sTf[cur][1];
      const uint32_t* offs = sOff[cur] + (td.blk_begin & 3);
      switch (h) {
        case 4: col_dispatch<4, INV, THREADS>(tf, a.params, buf, offs, a.out, nb, w); break;
        case 8: col_dispatch<8, INV, THREADS>(tf, a.params, buf, offs, a.out, nb, w); break;
        case 16: col_dispatch<16, INV, THREADS>(tf, a.params, buf, offs, a.out, nb, w); break;
        case 32: col_dispatch<32, INV, THREADS>(tf, a.params, buf, offs, a.out, nb, w); break;
        default: col_dispatch<64, INV, THREADS>(tf, a.params, buf, offs, a.out, nb, w); break;
      }
    }
    t = tn;
    tn = tn2;
    tn2 = tn3;
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
    for (int i = tid; i < kMaxRanges / 32; i += THREADS) a.sched->exhausted[i] = 0u;
    if (tid == 0) a.sched->done = 0u;
    __threadfence();
  }
}

}  // namespace adjtx
