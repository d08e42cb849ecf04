// Fused, persistent 2-D adjusted-transform kernels (forward and inverse).
//
// One CTA processes one tile at a time: a group of blocks that share
// (w, h, tf_h, tf_v).  Per tile:
//   1. stage the blocks' input samples into shared memory with 16-B cp.async copies
//      (coalesced global reads, bank-conflict-free padded rows);
//   2. row pass: one thread per block row applies the horizontal 1-D transform
//      (band -> core -> post, or the transposed chain for the inverse) in registers
//      and writes the row into the transpose buffer T;
//   3. column pass: one thread per block column reads its column of T, applies the
//      vertical 1-D transform and writes the outputs straight to global memory
//      (a warp covers consecutive columns, so each store instruction is coalesced).
// Tiles are taken from a global atomic counter; the last CTA to finish resets it, so
// a launch needs no separate reset.  No CTA ever waits for another one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_device.cuh"
#include "adjtx_kernels.h"

namespace adjtx {

template <int W, bool INV, int THREADS>
__device__ __forceinline__ void row_pass(const TfDev& tf, const float* __restrict__ P,
                                         const unsigned char* stg, float* sT, int nb, int h) {
  const int lgh = ilog2(h);
  const int nlines = nb * h;
  const int rs = stg_row_bytes(W, INV ? 4 : 2);
  const int tb = t_block_floats(W, h);
  for (int l = threadIdx.x; l < nlines; l += THREADS) {
    const int b = l >> lgh, r = l & (h - 1);
    DstTRow dst{sT + b * tb + r * (W + 1)};
    if constexpr (INV) {
      SrcRowF32 src{reinterpret_cast<const float*>(stg + l * rs)};
      line_transform<W, true>(tf, P, src, dst);
    } else {
      SrcRowI16 src{reinterpret_cast<const int16_t*>(stg + l * rs)};
      line_transform<W, false>(tf, P, src, dst);
    }
  }
}

template <int H, bool INV, int THREADS>
__device__ __forceinline__ void col_pass(const TfDev& tf, const float* __restrict__ P, const float* sT,
                                         const uint32_t* sOff, float* __restrict__ out, int nb, int w) {
  const int lgw = ilog2(w);
  const int nlines = nb * w;
  const int tb = t_block_floats(w, H);
  for (int l = threadIdx.x; l < nlines; l += THREADS) {
    const int b = l >> lgw, c = l & (w - 1);
    SrcTCol src{sT + b * tb + c, w + 1};
    DstGCol dst{out + (size_t)sOff[b] * 16 + c, w};
    line_transform<H, INV>(tf, P, src, dst);
  }
}

// Shared memory limits residency to kSmemCtasPerSm CTAs per SM; the register budget
// follows from that, so spills are never traded for occupancy that smem forbids.
constexpr int kSmemCtasPerSm = (227 * 1024) / (kSmemBytes + 2048);

template <bool INV, int THREADS>
__global__ void __launch_bounds__(THREADS, kSmemCtasPerSm * 64 / THREADS) fused_kernel(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* sT = reinterpret_cast<float*>(smem);
  unsigned char* sStg = smem + kTBytes;
  __shared__ uint32_t sOff[kMaxTileBlocks];
  __shared__ int sTile;
  constexpr int esz = INV ? 4 : 2;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) sTile = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int t = sTile;
    if (t >= a.n_tiles) break;
    const TileDev td = a.tiles[t];
    const int w = td.w, h = td.h, nb = td.nblk;
    for (int b = tid; b < nb; b += THREADS) sOff[b] = a.tile_blk[td.blk_begin + b];
    __syncthreads();

    // 1. stage the input tile
    {
      const int rowb = w * esz;
      const int rs = stg_row_bytes(w, esz);
      const int bstg = h * rs;
      const int lg_cpb = ilog2(w * h * esz / 16);      // 16-B chunks per block
      const int lg_cpr = rowb >= 16 ? ilog2(rowb / 16) : 0;
      const int total = nb << lg_cpb;
      const unsigned char* in = reinterpret_cast<const unsigned char*>(a.in);
      for (int g = tid; g < total; g += THREADS) {
        const int b = g >> lg_cpb, q = g & ((1 << lg_cpb) - 1);
        int d;
        if (rowb <= 16) d = q * 16;
        else d = (q >> lg_cpr) * rs + (q & ((1 << lg_cpr) - 1)) * 16;
        cp_async16(sStg + b * bstg + d, in + ((size_t)sOff[b] * 16 * esz) + q * 16);
      }
      cp_async_commit();
      cp_async_wait_all();
    }
    __syncthreads();

    // 2. row pass (horizontal transform, length w)
    {
      const TfDev tf = a.tfs[td.tf_h];
      switch (w) {
        case 4: row_pass<4, INV, THREADS>(tf, a.params, sStg, sT, nb, h); break;
        case 8: row_pass<8, INV, THREADS>(tf, a.params, sStg, sT, nb, h); break;
        case 16: row_pass<16, INV, THREADS>(tf, a.params, sStg, sT, nb, h); break;
        case 32: row_pass<32, INV, THREADS>(tf, a.params, sStg, sT, nb, h); break;
        default: row_pass<64, INV, THREADS>(tf, a.params, sStg, sT, nb, h); break;
      }
    }
    __syncthreads();

    // 3. column pass (vertical transform, length h), stores to global memory
    {
      const TfDev tf = a.tfs[td.tf_v];
      switch (h) {
        case 4: col_pass<4, INV, THREADS>(tf, a.params, sT, sOff, a.out, nb, w); break;
        case 8: col_pass<8, INV, THREADS>(tf, a.params, sT, sOff, a.out, nb, w); break;
        case 16: col_pass<16, INV, THREADS>(tf, a.params, sT, sOff, a.out, nb, w); break;
        case 32: col_pass<32, INV, THREADS>(tf, a.params, sT, sOff, a.out, nb, w); break;
        default: col_pass<64, INV, THREADS>(tf, a.params, sT, sOff, a.out, nb, w); break;
      }
    }
    __syncthreads();
  }

  // The last CTA out resets the work counter for the next launch on this plan.
  if (tid == 0) {
    __threadfence();
    const unsigned done = atomicAdd(a.counter + 1, 1u);
    if (done == gridDim.x - 1) {
      atomicExch(a.counter, 0u);
      atomicExch(a.counter + 1, 0u);
    }
  }
}

template <bool INV>
static const void* fused_fn(int threads) {
  switch (threads) {
    case 64: return reinterpret_cast<const void*>(&fused_kernel<INV, 64>);
    case 128: return reinterpret_cast<const void*>(&fused_kernel<INV, 128>);
    default: return nullptr;
  }
}

const void* fused_kernel_ptr(bool inverse, int threads) {
  return inverse ? fused_fn<true>(threads) : fused_fn<false>(threads);
}

cudaError_t launch_fused(bool inverse, int threads, int grid, const FusedArgs& args, cudaStream_t stream) {
  const void* fn = fused_kernel_ptr(inverse, threads);
  if (!fn) return cudaErrorInvalidValue;
  FusedArgs a = args;
  void* params[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, kSmemBytes, stream);
}

}  // namespace adjtx
