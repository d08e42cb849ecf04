// Device records and shared-memory layout rules, used by the host planner and the
// kernels alike.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define ADJ_HD __host__ __device__ __forceinline__ constexpr
#else
#define ADJ_HD constexpr inline
#endif

namespace adjtx {

enum { KIND_NONE = 0, KIND_BAND = 1, KIND_POST = 2, KIND_DENSE = 3 };

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
  uint32_t cs_off;    // float2 index of the first (cos, sin) pair (layers back to back)
  uint32_t q_off;     // float index of the kt x kt row-major padded Q (16-B aligned)
  int32_t k;          // post / dense: K (the unpadded size of Q); 0 otherwise
  uint32_t csl_off;   // float4 index of the per-layer table: layer l's (cos, sin) pairs at
                      // float4 csl_off + l * n / 4, two rotations a float4, an odd layer
                      // padded with one unused pair
  uint32_t qt_off;    // float index of the transpose of the padded Q (tile-wide forward post)
  uint32_t pad[3];
};
static_assert(sizeof(TfDev) == 64, "TfDev layout");

// A tile: blocks of one (w, h, tf_h, tf_v) class processed together by one CTA.
struct TileDev {
  uint32_t blk_begin;  // first entry in the tile block-offset list
  uint16_t nblk, w, h, tf_h, tf_v, pad;
};
static_assert(sizeof(TileDev) == 16, "TileDev layout");

// Shared memory of one CTA: two tile buffers (the tile being transformed and the next
// tile being loaded).  A tile holds at most kTileCoefs coefficients as FP32; the staged
// input of each row (int16 forward, FP32 inverse) sits inside that row's own region, so
// the row pass transforms it in place.
constexpr int kTileCoefs = 4096;
constexpr int kBufBytes = 4 * kTileCoefs;
constexpr int kSmemBytes = 2 * kBufBytes;
constexpr int kMaxTileBlocks = 256;
// Kernels whose input is int16 (the forward from residual blocks or frames) stage it into a
// separate int16 buffer and write the row pass's FP32 output into one tile buffer: 24 KB
// instead of 32 KB, which lets 8 CTAs share an SM.
constexpr int kStageI16Bytes = 2 * kTileCoefs;
constexpr int kSmemBytesI16 = kBufBytes + kStageI16Bytes;
// Shared memory of one GB300 SM, and what the hardware reserves for each resident CTA.
constexpr int kSmemPerSm = 228 * 1024;
constexpr int kSmemReservedPerCta = 1024;

// Work distribution.  The tile list is sorted by class, so consecutive tiles share
// (w, h, core, adjustment) and therefore code.  The planner cuts the list into up to
// kMaxRanges contiguous ranges of about equal work; the CTAs of SM s take tiles from range
// s mod n_ranges in order, so each SM walks through neighbouring classes and keeps its
// instruction cache warm.  A CTA whose range is used up moves to the range with the most
// unclaimed tiles (work stealing).  All words are zero between launches (the last CTA of a
// launch clears them).
constexpr int kMaxRanges = 256;
struct SchedState {
  unsigned pos[kMaxRanges];        // claims made on each range (tiles taken, plus failed claims)
  unsigned done;                   // CTAs finished
  unsigned pad[15];
};

ADJ_HD int ilog2(int x) {
  int r = 0;
  while ((1 << (r + 1)) <= x) ++r;
  return r;
}

// Tile buffer layout.  Block b of a tile starts at float b*w*h; row r of a block is w
// floats (w/4 chunks of 16 B) at r*w.  Chunk q of row r is stored at chunk slot q ^ f(r):
// 8 consecutive rows read or written with 16-B accesses then touch 8 distinct bank groups,
// and 32 consecutive columns of one row fall in 32 distinct banks.
ADJ_HD int sw_shift(int w) {
  const int lg = ilog2(w / 4);
  return lg >= 3 ? 0 : 3 - lg;
}
ADJ_HD int sw_mask(int w) { return (w / 4 < 8 ? w / 4 : 8) - 1; }
ADJ_HD int sw_f(int r, int w) { return (r >> sw_shift(w)) & sw_mask(w); }
// float index of element (r, c) inside a block of width w
ADJ_HD int sw_index(int r, int c, int w) { return r * w + ((((c >> 2) ^ sw_f(r, w))) << 2) + (c & 3); }

// Largest number of w x h blocks in one tile.
ADJ_HD int tile_capacity(int w, int h) {
  const int c = kTileCoefs / (w * h);
  return c < kMaxTileBlocks ? c : kMaxTileBlocks;
}

}  // namespace adjtx
