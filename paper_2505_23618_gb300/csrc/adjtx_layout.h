// Device records and shared-memory layout rules, used by the host planner and the
// kernels alike.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define ADJ_HD __host__ __device__ __forceinline__
#else
#define ADJ_HD inline
#endif

namespace adjtx {

enum { KIND_NONE = 0, KIND_BAND = 1, KIND_POST = 2 };

// One 1-D transform as the kernels see it (parameters live in one FP32 buffer).
struct TfDev {
  int32_t n;          // line length
  int32_t core;       // 0 DCT-2, 1 DCT-3, 2 DST-2, 3 DST-3
  int32_t kind;       // KIND_*
  int32_t n_layers;   // band layers
  int32_t n_pairs;    // total rotations over all layers
  int32_t kt;         // post: padded block size (power of two, 4 <= kt <= n)
  uint32_t par_lo;    // bit l = parity of layer l (l < 32)
  uint32_t par_hi;    // bit l-32 = parity of layer l (32 <= l < 64)
  uint32_t cs_off;    // float2 index of the first (cos, sin) pair
  uint32_t q_off;     // float index of the kt x kt row-major padded Q (16-B aligned)
  uint32_t pad0, pad1;
};
static_assert(sizeof(TfDev) == 48, "TfDev layout");

// A tile: blocks of one (w, h, tf_h, tf_v) class processed together by one CTA.
struct TileDev {
  uint32_t blk_begin;  // first entry in the tile block-offset list
  uint16_t nblk, w, h, tf_h, tf_v, pad;
};
static_assert(sizeof(TileDev) == 16, "TileDev layout");

// Shared-memory budgets of one CTA: the transpose buffer T (FP32) and the staging
// buffer of the input tile (int16 forward, FP32 inverse).  One 64x64 block fills both.
constexpr int kTBytes = 4 * 64 * 65;        // 16640
constexpr int kStgBytes = 64 * (4 * 64 + 16);  // 17408
constexpr int kSmemBytes = kTBytes + kStgBytes;
constexpr int kMaxTileBlocks = 256;

ADJ_HD int ilog2(int x) {
  int r = 0;
  while ((1 << (r + 1)) <= x) ++r;
  return r;
}

// Staging row stride in bytes: rows of 16 B or less are packed; longer rows get 16 B
// of padding so that 8 consecutive rows read with 16-B loads hit 8 distinct bank groups.
ADJ_HD int stg_row_bytes(int w, int esz) {
  const int rb = w * esz;
  return rb <= 16 ? rb : rb + 16;
}
ADJ_HD int stg_block_bytes(int w, int h, int esz) { return h * stg_row_bytes(w, esz); }

// T: each block row has w+1 floats (odd stride -> row-pass stores conflict-free);
// tall narrow blocks get w floats of block padding so that the blocks sharing a warp in
// the column pass fall into different bank windows.
ADJ_HD int t_block_floats(int w, int h) {
  return h * (w + 1) + ((w < 32 && h > w) ? w : 0);
}

// Largest number of blocks of size w x h that one tile can hold.
ADJ_HD int tile_capacity(int w, int h) {
  int a = kTBytes / (4 * t_block_floats(w, h));
  int b = kStgBytes / stg_block_bytes(w, h, 4);
  int c = a < b ? a : b;
  return c < kMaxTileBlocks ? c : kMaxTileBlocks;
}

}  // namespace adjtx
