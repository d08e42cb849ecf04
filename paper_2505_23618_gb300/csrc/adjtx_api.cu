// C ABI of the adjusted-transform library: plan creation, validation, parameter
// materialisation, tiling and the transform entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "adjtx.h"
#include "adjtx_kernels.h"

using namespace adjtx;

namespace {

// Message of the calling thread's last failed call.  A fixed buffer: reporting an error
// never allocates.
thread_local char g_err[512];

void clear_error() { g_err[0] = '\0'; }

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

// Maps the C++ exception in flight (a failed host allocation, in practice) to an error code.
// Called from the catch-all handler of every entry point that allocates host memory, so that
// no exception crosses the C ABI.
int entry_exception() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return fail(ADJ_ERR_NO_MEMORY, "host memory allocation failed");
  } catch (const std::exception& e) {
    return fail(ADJ_ERR_NO_MEMORY, "host allocation: %s", e.what());
  } catch (...) {
    return fail(ADJ_ERR_NO_MEMORY, "unknown C++ exception");
  }
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(ADJ_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

bool is_size(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64; }

int pairs_in_layer(int n, int parity) { return parity ? n / 2 - 1 : n / 2; }

struct TfHost {
  int n, core, kind, n_layers, k, kt, n_pairs;
  std::vector<uint8_t> parity;
  std::vector<double> angles;
  std::vector<double> q;  // k x k
};

// Host-buffer path: the offset-sorted block list is cut into chunks of up to about
// kHostChunkCoefs coefficients (about kMaxHostChunks of them for large lists, plus short ramp
// chunks at both ends); chunk c's input copy, kernel and output copy run on three streams, so
// copies of one chunk overlap the kernel and copies of others.
constexpr int64_t kHostChunkCoefs = 4 << 20;
constexpr int kMaxHostChunks = 16;
struct HostChunk {
  int64_t begin, end;   // samples [begin, end) covered by the chunk's blocks
  int tile0, n_tiles;   // the chunk's tiles in the host tile list
  int r0, n_ranges;     // its per-SM ranges in the host range list
};

}  // namespace

struct adj_plan {
  int device = 0;
  int n_sm = 0;
  int threads = 64;
  std::vector<TfHost> tfs;
  TfDev* d_tfs = nullptr;
  float* d_params = nullptr;
  size_t n_params = 0;
  bool has_blocks = false;
  int64_t n_blocks = 0;
  int64_t total = 0;
  TileDev* d_tiles = nullptr;
  uint32_t* d_tile_blk = nullptr;
  int n_tiles = 0;
  SchedState* d_sched = nullptr;  // [0] forward, [1] inverse, [2] Multiple forward
  unsigned* d_range_begin = nullptr;
  int n_ranges = 0;
  int grid_fwd = 0, grid_inv = 0;
  void* d_host_in = nullptr;
  float* d_host_out = nullptr;
  size_t host_cap = 0;
  PlainBlock* d_plain = nullptr;       // plain form: blocks grouped by size
  std::vector<PlainClass> plain;
  // backward: accumulator and gradient layouts per transform, scratch
  std::vector<int> m_off, g_off, kq;
  int P = 0, n_grad = 0;
  int* d_layout = nullptr;             // m_off | g_off | kq on the device
  float* d_partial = nullptr;
  double* d_M = nullptr;
  int bwd_grid = 0;
  std::vector<adj_block_t> blocks;     // validated, in storage order
  std::vector<int64_t> orig;           // caller's index of each entry of `blocks`
  // Multiple forward: prepared block list, side offsets in the caller's block order
  bool multi = false;
  std::vector<int64_t> side_off;
  // Blocks inside a frame: frame offsets (y * stride + x) in the caller's block order
  bool frame = false;
  int32_t frame_w = 0, frame_h = 0, frame_stride = 0;
  std::vector<int64_t> frame_off;
  uint32_t* d_tile_side = nullptr;     // side or frame offset / 4, parallel to d_tile_blk
  int occ_multi = 0, grid_multi = 0;
  int occ_frame = 0, grid_frame = 0;          // frame inverses (FP32 and int16 output)
  int occ_frame_fwd = 0, grid_frame_fwd = 0;  // frame forward
  int occ_f32 = 0, grid_f32 = 0;      // forward of FP32 blocks
  adj_tuning_t tuning{};
  int occ_fwd = 0, occ_inv = 0;        // resident CTAs per SM of the fused kernels
  // host-buffer path (built on first use, dropped with the block layout)
  std::vector<HostChunk> chunks;
  bool chunks_valid = false;
  TileDev* d_ctiles = nullptr;
  uint32_t* d_ctile_blk = nullptr;
  unsigned* d_crange = nullptr;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_k;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

namespace {

int validate_tf(const adj_1d_desc_t& d, int idx, TfHost* out) {
  if (!is_size(d.n)) return fail(ADJ_ERR_UNSUPPORTED_SIZE, "tf %d: n=%d not in {4,8,16,32,64}", idx, d.n);
  if (d.core < 0 || d.core > 3) return fail(ADJ_ERR_INVALID_ARG, "tf %d: core %d", idx, d.core);
  if (d.kind < 0 || d.kind > 3) return fail(ADJ_ERR_INVALID_ARG, "tf %d: kind %d", idx, d.kind);
  if (d.kind == ADJ_ADJ_DENSE && d.k != d.n)
    return fail(ADJ_ERR_PARAM_MISMATCH, "tf %d: a dense transform needs k = n (%d, %d)", idx, d.k, d.n);
  TfHost t{};
  t.n = d.n;
  t.core = d.core;
  t.kind = d.kind;
  if (d.kind == ADJ_ADJ_PRE_BAND) {
    if (d.n_layers < 0 || d.n_layers > ADJ_MAX_LAYERS)
      return fail(ADJ_ERR_UNSUPPORTED_SIZE, "tf %d: %d layers (max %d)", idx, d.n_layers, ADJ_MAX_LAYERS);
    if (d.n_layers > 0 && !d.layer_parity) return fail(ADJ_ERR_INVALID_ARG, "tf %d: null layer_parity", idx);
    t.n_layers = d.n_layers;
    int np = 0;
    for (int l = 0; l < d.n_layers; ++l) {
      if (d.layer_parity[l] > 1) return fail(ADJ_ERR_INVALID_ARG, "tf %d: parity of layer %d is %d", idx, l, d.layer_parity[l]);
      t.parity.push_back(d.layer_parity[l]);
      np += pairs_in_layer(d.n, d.layer_parity[l]);
    }
    if (np > 0 && !d.angles) return fail(ADJ_ERR_INVALID_ARG, "tf %d: null angles", idx);
    t.n_pairs = np;
    t.angles.assign(d.angles, d.angles + np);
    for (double a : t.angles)
      if (!std::isfinite(a)) return fail(ADJ_ERR_PARAM_MISMATCH, "tf %d: non-finite angle", idx);
  } else if (d.kind == ADJ_ADJ_POST_BLOCK || d.kind == ADJ_ADJ_DENSE) {
    if (d.k < 1 || d.k > d.n) return fail(ADJ_ERR_UNSUPPORTED_SIZE, "tf %d: K=%d with n=%d", idx, d.k, d.n);
    if (!d.q) return fail(ADJ_ERR_INVALID_ARG, "tf %d: null q", idx);
    t.k = d.k;
    int kt = 4;
    while (kt < d.k) kt *= 2;
    t.kt = kt;
    t.q.assign(d.q, d.q + (size_t)d.k * d.k);
    double worst = 0.0;
    for (int i = 0; i < d.k; ++i)
      for (int j = 0; j < d.k; ++j) {
        double s = 0.0;
        for (int r = 0; r < d.k; ++r) s += t.q[r * d.k + i] * t.q[r * d.k + j];
        if (!std::isfinite(s)) return fail(ADJ_ERR_PARAM_MISMATCH, "tf %d: non-finite Q", idx);
        worst = std::max(worst, std::fabs(s - (i == j ? 1.0 : 0.0)));
      }
    if (worst > 1e-6) return fail(ADJ_ERR_PARAM_MISMATCH, "tf %d: Q not orthogonal (|Q^T Q - I| = %g)", idx, worst);
  }
  *out = std::move(t);
  return ADJ_OK;
}

// FP64 -> FP32 parameter materialisation (cos/sin of every angle; padded Q).
void materialise(const std::vector<TfHost>& tfs, std::vector<float>* params, std::vector<TfDev>* devs) {
  params->clear();
  devs->clear();
  for (const TfHost& t : tfs) {
    TfDev d{};
    d.n = t.n;
    d.core = t.core;
    d.kind = t.kind;
    if (t.kind == ADJ_ADJ_PRE_BAND) {
      d.n_layers = t.n_layers;
      d.n_pairs = t.n_pairs;
      for (int l = 0; l < t.n_layers; ++l) {
        if (t.parity[l]) {
          if (l < 32) d.par_lo |= 1u << l;
          else d.par_hi |= 1u << (l - 32);
        }
      }
      if (params->size() % 2) params->push_back(0.f);
      d.cs_off = (uint32_t)(params->size() / 2);
      for (double a : t.angles) {
        params->push_back((float)std::cos(a));
        params->push_back((float)std::sin(a));
      }
      // per-layer table of the kernels: n / 2 pairs a layer, 16-byte aligned
      while (params->size() % 4) params->push_back(0.f);
      d.csl_off = (uint32_t)(params->size() / 4);
      for (int l = 0, a = 0; l < t.n_layers; ++l) {
        const int np = pairs_in_layer(t.n, t.parity[l]);
        for (int j = 0; j < t.n / 2; ++j) {
          params->push_back(j < np ? (float)std::cos(t.angles[a + j]) : 1.f);
          params->push_back(j < np ? (float)std::sin(t.angles[a + j]) : 0.f);
        }
        a += np;
      }
    } else if (t.kind == ADJ_ADJ_POST_BLOCK || t.kind == ADJ_ADJ_DENSE) {
      d.kt = t.kt;
      d.k = t.k;
      while (params->size() % 4) params->push_back(0.f);
      d.q_off = (uint32_t)params->size();
      for (int i = 0; i < t.kt; ++i)
        for (int j = 0; j < t.kt; ++j) {
          double v = (i < t.k && j < t.k) ? t.q[i * t.k + j] : (i == j ? 1.0 : 0.0);
          params->push_back((float)v);
        }
    }
    devs->push_back(d);
  }
  // transposes of the padded Q blocks (tile-wide forward post block), after all other tables so
  // that those stay packed together
  for (size_t n = 0; n < tfs.size(); ++n) {
    const TfHost& t = tfs[n];
    if (t.kind != ADJ_ADJ_POST_BLOCK && t.kind != ADJ_ADJ_DENSE) continue;
    while (params->size() % 4) params->push_back(0.f);
    (*devs)[n].qt_off = (uint32_t)params->size();
    for (int j = 0; j < t.kt; ++j)
      for (int i = 0; i < t.kt; ++i) {
        double v = (i < t.k && j < t.k) ? t.q[i * t.k + j] : (i == j ? 1.0 : 0.0);
        params->push_back((float)v);
      }
  }
  while (params->size() % 4) params->push_back(0.f);
  if (params->empty()) params->resize(4, 0.f);
}

// Uploads the tables of `tfs` (the plan's transforms, or their replacement).
int upload_params(adj_plan* p, const std::vector<TfHost>& tfs) {
  std::vector<float> params;
  std::vector<TfDev> devs;
  materialise(tfs, &params, &devs);
  if (!p->d_params) {
    CUDA_TRY(cudaMalloc(&p->d_params, params.size() * sizeof(float)));
    CUDA_TRY(cudaMalloc(&p->d_tfs, std::max<size_t>(1, devs.size()) * sizeof(TfDev)));
    p->n_params = params.size();
  } else if (params.size() != p->n_params) {
    return fail(ADJ_ERR_PARAM_MISMATCH, "parameter size changed");
  }
  CUDA_TRY(cudaMemcpy(p->d_params, params.data(), params.size() * sizeof(float), cudaMemcpyHostToDevice));
  if (!devs.empty())
    CUDA_TRY(cudaMemcpy(p->d_tfs, devs.data(), devs.size() * sizeof(TfDev), cudaMemcpyHostToDevice));
  return ADJ_OK;
}

void free_chunks(adj_plan* p) {
  cudaFree(p->d_ctiles);
  cudaFree(p->d_ctile_blk);
  cudaFree(p->d_crange);
  p->d_ctiles = nullptr;
  p->d_ctile_blk = nullptr;
  p->d_crange = nullptr;
  p->chunks.clear();
  p->chunks_valid = false;
}

void free_blocks(adj_plan* p) {
  free_chunks(p);
  cudaFree(p->d_tiles);
  cudaFree(p->d_tile_blk);
  cudaFree(p->d_range_begin);
  cudaFree(p->d_plain);
  cudaFree(p->d_tile_side);
  p->d_tile_side = nullptr;
  p->d_plain = nullptr;
  p->plain.clear();
  p->d_tiles = nullptr;
  p->d_tile_blk = nullptr;
  p->d_range_begin = nullptr;
  p->n_ranges = 0;
  p->n_tiles = 0;
  p->has_blocks = false;
}

int check_ptr(const void* ptr, const char* name) {
  if (!ptr) return fail(ADJ_ERR_INVALID_ARG, "%s is null", name);
  if (reinterpret_cast<uintptr_t>(ptr) % 16) return fail(ADJ_ERR_MISALIGNED, "%s is not 16-byte aligned", name);
  return ADJ_OK;
}

int run(adj_plan* p, bool inverse, const void* in, float* out, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(in, "input")) || (rc = check_ptr(out, "output"))) return rc;
  if (p->n_tiles == 0) return ADJ_OK;
  FusedArgs a{};
  a.tiles = p->d_tiles;
  a.tile_blk = p->d_tile_blk;
  a.tfs = p->d_tfs;
  a.params = p->d_params;
  a.in = in;
  a.out = out;
  a.sched = p->d_sched + (inverse ? 1 : 0);
  a.range_begin = p->d_range_begin;
  a.n_tiles = p->n_tiles;
  a.n_ranges = p->n_ranges;
  cudaError_t e = launch_fused(inverse, p->threads, inverse ? p->grid_inv : p->grid_fwd, a, stream);
  if (e != cudaSuccess) return cuda_fail(e, inverse ? "inverse launch" : "forward launch");
  return ADJ_OK;
}

// Forward of packed FP32 blocks: the fused kernel with FP32 staging, on the forward's tiles.
int run_fwd_f32(adj_plan* p, const float* in, float* out, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(in, "input")) || (rc = check_ptr(out, "output"))) return rc;
  if (p->n_tiles == 0) return ADJ_OK;
  FusedArgs a{};
  a.tiles = p->d_tiles;
  a.tile_blk = p->d_tile_blk;
  a.tfs = p->d_tfs;
  a.params = p->d_params;
  a.in = in;
  a.out = out;
  a.sched = p->d_sched;
  a.range_begin = p->d_range_begin;
  a.n_tiles = p->n_tiles;
  a.n_ranges = p->n_ranges;
  cudaError_t e = launch_fwd_f32(p->grid_f32, a, stream);
  if (e != cudaSuccess) return cuda_fail(e, "FP32 forward launch");
  return ADJ_OK;
}

int run_multi(adj_plan* p, const int16_t* in, float* out, float* side, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  if (!p->multi) return fail(ADJ_ERR_INVALID_ARG, "adj_plan_prepare_multiple has not been called for this block list");
  int rc;
  if ((rc = check_ptr(in, "input")) || (rc = check_ptr(out, "output"))) return rc;
  if (p->side_off.back() > 0 && (rc = check_ptr(side, "side buffer"))) return rc;
  if (p->n_tiles == 0) return ADJ_OK;
  FusedArgs a{};
  a.tiles = p->d_tiles;
  a.tile_blk = p->d_tile_blk;
  a.tfs = p->d_tfs;
  a.params = p->d_params;
  a.in = in;
  a.out = out;
  a.sched = p->d_sched + 2;
  a.range_begin = p->d_range_begin;
  a.n_tiles = p->n_tiles;
  a.n_ranges = p->n_ranges;
  a.side = side;
  a.tile_aux = p->d_tile_side;
  cudaError_t e = launch_multi(p->grid_multi, a, stream);
  if (e != cudaSuccess) return cuda_fail(e, "Multiple forward launch");
  return ADJ_OK;
}

int run_frame(adj_plan* p, bool inverse, const void* in, void* out, bool i16, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "no block list");
  if (!p->frame) return fail(ADJ_ERR_INVALID_ARG, "the plan's blocks were not given with adj_plan_set_frame_blocks");
  int rc;
  if ((rc = check_ptr(in, "input")) || (rc = check_ptr(out, "output"))) return rc;
  if (p->n_tiles == 0) return ADJ_OK;
  FusedArgs a{};
  a.tiles = p->d_tiles;
  a.tile_blk = p->d_tile_blk;
  a.tfs = p->d_tfs;
  a.params = p->d_params;
  a.in = in;
  a.out = static_cast<float*>(out);
  a.sched = p->d_sched + (inverse ? 1 : 0);
  a.range_begin = p->d_range_begin;
  a.n_tiles = p->n_tiles;
  a.n_ranges = p->n_ranges;
  a.tile_aux = p->d_tile_side;
  a.frame_stride = p->frame_stride;
  cudaError_t e = launch_frame(inverse, i16, inverse ? p->grid_frame : p->grid_frame_fwd, a, stream);
  if (e != cudaSuccess) return cuda_fail(e, "frame launch");
  return ADJ_OK;
}

int run_bwd(adj_plan* p, const void* x, bool x_f32, const float* gy, float* gx, float* gparams, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(x, "input")) || (rc = check_ptr(gy, "output gradient"))) return rc;
  if (gx && (rc = check_ptr(gx, "input gradient"))) return rc;
  if (gparams && (rc = check_ptr(gparams, "parameter gradient"))) return rc;
  if (p->n_tiles == 0) {
    if (gparams && p->n_grad) CUDA_TRY(cudaMemsetAsync(gparams, 0, p->n_grad * sizeof(float), stream));
    return ADJ_OK;
  }
  if (!p->bwd_grid) {
    const void* fn = bwd_kernel_ptr(true);
    const void* fn2 = bwd_kernel_ptr(false);
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bwd_smem_bytes()));
    CUDA_TRY(cudaFuncSetAttribute(fn2, cudaFuncAttributeMaxDynamicSharedMemorySize, bwd_smem_bytes()));
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBwdThreads, bwd_smem_bytes()));
    p->bwd_grid = std::max(1, occ) * p->n_sm;
  }
  const int grid = std::min(p->bwd_grid, p->n_tiles);
  if (!p->d_partial && p->P) {
    CUDA_TRY(cudaMalloc(&p->d_partial, (size_t)p->bwd_grid * p->P * sizeof(float)));
    CUDA_TRY(cudaMalloc(&p->d_M, (size_t)p->P * sizeof(double)));
  }
  BwdArgs a{};
  a.tiles = p->d_tiles;
  a.tile_blk = p->d_tile_blk;
  a.tfs = p->d_tfs;
  a.params = p->d_params;
  a.x = x;
  a.gy = gy;
  a.gx = gx;
  a.partial = p->d_partial;
  a.m_off = p->d_layout;
  a.n_tiles = p->n_tiles;
  a.P = p->P;
  const int n = (int)p->tfs.size();
  cudaError_t e = launch_bwd(!x_f32, grid, a, p->d_M, p->d_tfs, n, p->d_layout, p->d_layout + n, p->d_layout + 2 * n,
                             gparams, stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return ADJ_OK;
}

int run_plain(adj_plan* p, bool inverse, const void* in, float* out, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(in, "input")) || (rc = check_ptr(out, "output"))) return rc;
  cudaError_t e = launch_plain(inverse, p->plain.data(), (int)p->plain.size(), p->d_tfs, p->d_params, in, out, stream);
  if (e != cudaSuccess) return cuda_fail(e, "plain-form launch");
  return ADJ_OK;
}

int ensure_host_staging(adj_plan* p) {
  const size_t need = (size_t)std::max<int64_t>(p->total, 4) * sizeof(float);
  if (p->host_cap >= need) return ADJ_OK;
  cudaFree(p->d_host_in);
  cudaFree(p->d_host_out);
  p->d_host_in = nullptr;
  p->d_host_out = nullptr;
  p->host_cap = 0;
  CUDA_TRY(cudaMalloc(&p->d_host_in, need));
  CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&p->d_host_out), need));
  CUDA_TRY(cudaMemset(p->d_host_out, 0, need));
  p->host_cap = need;
  return ADJ_OK;
}

}  // namespace

int tuned_capacity(const adj_plan* p, int w, int h) {
  const int cls = (ilog2(w) - 2) * 5 + (ilog2(h) - 2);
  const int div = std::max(1, p->tuning.cap_div[cls]);
  return std::max(1, tile_capacity(w, h) / div);
}

void apply_grid(adj_plan* p) {
  const int c = p->tuning.ctas_per_sm;
  p->grid_fwd = std::max(1, c > 0 ? std::min(c, p->occ_fwd) : p->occ_fwd) * p->n_sm;
  p->grid_inv = std::max(1, c > 0 ? std::min(c, p->occ_inv) : p->occ_inv) * p->n_sm;
  p->grid_multi = std::max(1, c > 0 ? std::min(c, p->occ_multi) : p->occ_multi) * p->n_sm;
  p->grid_frame = std::max(1, c > 0 ? std::min(c, p->occ_frame) : p->occ_frame) * p->n_sm;
  p->grid_frame_fwd = std::max(1, c > 0 ? std::min(c, p->occ_frame_fwd) : p->occ_frame_fwd) * p->n_sm;
  p->grid_f32 = std::max(1, c > 0 ? std::min(c, p->occ_f32) : p->occ_f32) * p->n_sm;
}

// Tiles, per-SM ranges and the plain form's per-size lists for the plan's block list,
// under the plan's tuning.
// Host image of a tile list: tiles, their block offsets (and Multiple side offsets) and
// the per-SM ranges.  blk_begin indexes tblk; range entries index tiles.
struct TileSet {
  std::vector<TileDev> tiles;
  std::vector<uint32_t> tblk, tside;
  std::vector<unsigned> rbeg;
  int n_ranges = 0;
};

// Default share (percent of the estimated cost) of the cheapest tiles that are dealt over the
// ends of the per-SM ranges (adj_tuning_t::tail_pct).
constexpr int kDefaultTailPct = 10;

// Estimated run time of a tile in the fused kernel (microseconds on GB300 at 6 CTAs per SM),
// a least-squares fit of measured tile times on a mixed workload: a fixed cost per tile;
// per line, an extra cost for 64-sample lines (one line per thread, no packed pairs) and for
// 4-sample rows; and the band rotations (n x layers per line) and post-block products (kt^2
// per line) of each direction.  The fast cores, loads and stores of shorter lines cost about
// the same per sample and fold into the fixed part.  Per-SM ranges are balanced on this
// cost, so that every SM runs out of its own tiles at about the same time.
double tile_cost(const adj_plan* p, const TileDev& t) {
  auto adjust = [](const TfHost& f) {
    if (f.kind == KIND_BAND) return 1.3e-4 * f.n * f.n_layers;
    if (f.kind == KIND_POST || f.kind == KIND_DENSE) return 1.0e-4 * f.kt * f.kt;
    return 0.0;
  };
  auto row = [&](const TfHost& f) { return (f.n == 64 ? 0.018 : f.n == 4 ? 0.0045 : 0.0) + adjust(f); };
  auto col = [&](const TfHost& f) { return (f.n == 64 ? 0.021 : 0.0) + adjust(f); };
  const double lines_h = (double)t.nblk * t.h, lines_v = (double)t.nblk * t.w;
  return 6.3 + lines_h * row(p->tfs[t.tf_h]) + lines_v * col(p->tfs[t.tf_v]);
}

// Tiles of the blocks [i0, i1) of the plan's (offset-sorted) list: blocks of one
// (w, h, tf_h, tf_v) class, filled in storage order, then listed class by class so that
// consecutive tiles run the same code (by block size, then by the code-determining
// (core, kind) of each direction, then by transform index); then per-SM ranges of about
// equal estimated cost (tile_cost), each ordered most expensive tile first.  Block offsets
// are appended to ts->tblk (4-aligned lists).
void build_tiles(const adj_plan* p, size_t i0, size_t i1, TileSet* ts) {
  struct Open {
    std::vector<uint32_t> offs, sides;
    int64_t first;
  };
  std::unordered_map<uint64_t, Open> open;
  struct Done {
    uint64_t key;
    int64_t first;
    TileDev t;
    std::vector<uint32_t> offs, sides;
  };
  std::vector<Done> done;
  auto emit = [&](uint64_t key, Open& o) {
    Done d;
    d.key = key;
    d.first = o.first;
    d.t = TileDev{};
    d.t.w = (uint16_t)(key >> 48);
    d.t.h = (uint16_t)(key >> 32);
    d.t.tf_h = (uint16_t)(key >> 16);
    d.t.tf_v = (uint16_t)key;
    d.t.nblk = (uint16_t)o.offs.size();
    d.offs.swap(o.offs);
    d.sides.swap(o.sides);
    done.push_back(std::move(d));
  };
  for (size_t i = i0; i < i1; ++i) {
    const adj_block_t& b = p->blocks[i];
    const uint64_t key = ((uint64_t)b.w << 48) | ((uint64_t)b.h << 32) | ((uint64_t)b.tf_h << 16) | b.tf_v;
    Open& o = open[key];
    if (o.offs.empty()) o.first = b.offset;
    o.offs.push_back((uint32_t)(b.offset / 16));
    if (p->multi) o.sides.push_back((uint32_t)(p->side_off[p->orig[i]] / 4));
    else if (p->frame) o.sides.push_back((uint32_t)(p->frame_off[p->orig[i]] / 4));
    if ((int)o.offs.size() >= tuned_capacity(p, b.w, b.h)) emit(key, o);
  }
  for (auto& kv : open)
    if (!kv.second.offs.empty()) emit(kv.first, kv.second);
  auto code_key = [&](const Done& d) {
    const TfHost &th = p->tfs[d.t.tf_h], &tv = p->tfs[d.t.tf_v];
    return ((uint64_t)d.t.w << 40) | ((uint64_t)d.t.h << 32) | ((uint64_t)th.kind << 28) |
           ((uint64_t)th.core << 24) | ((uint64_t)tv.kind << 20) | ((uint64_t)tv.core << 16);
  };
  std::stable_sort(done.begin(), done.end(), [&](const Done& a, const Done& b) {
    const uint64_t ka = code_key(a), kb = code_key(b);
    if (ka != kb) return ka < kb;
    return a.key != b.key ? a.key < b.key : a.first < b.first;
  });
  std::vector<TileDev>& tiles = ts->tiles;
  std::vector<uint32_t>& tblk = ts->tblk;
  std::vector<uint32_t>& tside = ts->tside;
  const size_t first_tile = tiles.size();
  tiles.reserve(first_tile + done.size());
  tblk.reserve(tblk.size() + (i1 - i0) + 4);
  // Each tile's block list starts on a 16-byte boundary and the list ends with 4 spare
  // entries: the kernel fetches a tile's offsets with 16-byte asynchronous copies.  The
  // side offsets of the Multiple form follow the same indexing.
  for (Done& d : done) {
    while (tblk.size() % 4) tblk.push_back(0u);
    d.t.blk_begin = (uint32_t)tblk.size();
    tiles.push_back(d.t);
    tblk.insert(tblk.end(), d.offs.begin(), d.offs.end());
    if (p->multi || p->frame) {
      tside.resize(d.t.blk_begin, 0u);
      tside.insert(tside.end(), d.sides.begin(), d.sides.end());
    }
  }
  tblk.resize(tblk.size() + 4, 0u);
  if (p->multi || p->frame) tside.resize(tblk.size(), 0u);

  // Per-SM ranges of this set's tiles (indices relative to its first tile) with about
  // equal estimated cost.
  const size_t nt = tiles.size() - first_tile;
  const int n_ranges = nt == 0 ? 0 : (int)std::min<size_t>({(size_t)std::max(1, p->n_sm * std::max(1, p->tuning.ranges_per_sm)), (size_t)kMaxRanges, nt});
  std::vector<unsigned>& rbeg = ts->rbeg;
  const size_t r0 = rbeg.size();  // this set's first range entry (ts may hold earlier sets)
  if (n_ranges > 0) {
    // The cheapest tiles, tail_pct percent of the estimated cost, are dealt over the ends of
    // all ranges: whichever tiles a CTA still holds when the work runs out are then short
    // ones, whatever classes its range holds.  The other tiles are cut into ranges in class
    // order.  Both parts are cut on their cumulative cost.
    std::vector<double> cost(nt);
    double total = 0.0;
    for (size_t i = 0; i < nt; ++i) total += (cost[i] = tile_cost(p, tiles[first_tile + i]));
    std::vector<char> in_tail(nt, 0);
    if (p->tuning.tail_pct > 0) {
      std::vector<size_t> by_cost(nt);
      for (size_t i = 0; i < nt; ++i) by_cost[i] = i;
      std::stable_sort(by_cost.begin(), by_cost.end(), [&](size_t x, size_t y) { return cost[x] < cost[y]; });
      const double budget = total * p->tuning.tail_pct / 100.0;
      double acc = 0.0;
      for (size_t i : by_cost) {
        if (acc + cost[i] > budget) break;
        acc += cost[i];
        in_tail[i] = 1;
      }
    }
    std::vector<size_t> part[2];
    for (size_t i = 0; i < nt; ++i) part[in_tail[i]].push_back(i);
    // range boundaries of each part, cut on the part's cumulative cost
    std::vector<size_t> bounds[2];
    for (int q = 0; q < 2; ++q) {
      const std::vector<size_t>& idx = part[q];
      std::vector<double> cum(idx.size() + 1, 0.0);
      for (size_t i = 0; i < idx.size(); ++i) cum[i + 1] = cum[i] + cost[idx[i]];
      bounds[q].push_back(0);
      for (int r = 1; r < n_ranges; ++r) {
        const size_t i = std::lower_bound(cum.begin(), cum.end(), cum.back() * r / n_ranges) - cum.begin();
        bounds[q].push_back(std::max(bounds[q].back(), std::min(i, idx.size())));
      }
      bounds[q].push_back(idx.size());
    }
    std::vector<TileDev> order;
    order.reserve(nt);
    rbeg.push_back(0);
    for (int r = 0; r < n_ranges; ++r) {
      for (int q = 0; q < 2; ++q)
        for (size_t i = bounds[q][r]; i < bounds[q][r + 1]; ++i) order.push_back(tiles[first_tile + part[q][i]]);
      rbeg.push_back((unsigned)order.size());
    }
    std::copy(order.begin(), order.end(), tiles.begin() + first_tile);
  }
  // Within each range the most expensive tiles go first (ties keep the class order), so the
  // tiles still queued when the ranges run dry are the short ones.
  for (int r = 0; r < n_ranges; ++r) {
    auto b = tiles.begin() + first_tile + rbeg[r0 + r], e = tiles.begin() + first_tile + rbeg[r0 + r + 1];
    std::stable_sort(b, e, [&](const TileDev& x, const TileDev& y) { return tile_cost(p, x) > tile_cost(p, y); });
  }
  ts->n_ranges = n_ranges;
}

// Tiles, per-SM ranges and the plain form's per-size lists for the plan's block list,
// under the plan's tuning.
int build_layout(adj_plan* p) {
  TileSet ts;
  build_tiles(p, 0, p->blocks.size(), &ts);
  const std::vector<TileDev>& tiles = ts.tiles;
  const std::vector<uint32_t>& tblk = ts.tblk;
  const std::vector<uint32_t>& tside = ts.tside;
  const std::vector<unsigned>& rbeg = ts.rbeg;
  const int n_ranges = ts.n_ranges;

  // Plain form: blocks grouped by size, in storage order within a size.
  std::vector<PlainBlock> pblk;
  std::vector<PlainClass> pcls;
  for (int lw = 2; lw <= 6; ++lw)
    for (int lh = 2; lh <= 6; ++lh) {
      PlainClass c{1 << lw, 1 << lh, 0, nullptr};
      const size_t first = pblk.size();
      for (const adj_block_t& b : p->blocks) {
        if (b.w == c.w && b.h == c.h) pblk.push_back(PlainBlock{(uint32_t)(b.offset / 16), b.tf_h, b.tf_v});
      }
      c.n_blocks = (int)(pblk.size() - first);
      c.blocks = reinterpret_cast<const PlainBlock*>(first);  // index for now, pointer after upload
      if (c.n_blocks) pcls.push_back(c);
    }

  free_blocks(p);
  if (!pblk.empty()) {
    CUDA_TRY(cudaMalloc(&p->d_plain, pblk.size() * sizeof(PlainBlock)));
    CUDA_TRY(cudaMemcpy(p->d_plain, pblk.data(), pblk.size() * sizeof(PlainBlock), cudaMemcpyHostToDevice));
    for (PlainClass& c : pcls) c.blocks = p->d_plain + reinterpret_cast<size_t>(c.blocks);
  }
  p->plain = pcls;
  if (!tiles.empty()) {
    CUDA_TRY(cudaMalloc(&p->d_tiles, tiles.size() * sizeof(TileDev)));
    CUDA_TRY(cudaMalloc(&p->d_tile_blk, tblk.size() * sizeof(uint32_t)));
    CUDA_TRY(cudaMalloc(&p->d_range_begin, rbeg.size() * sizeof(unsigned)));
    CUDA_TRY(cudaMemcpy(p->d_tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->d_tile_blk, tblk.data(), tblk.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->d_range_begin, rbeg.data(), rbeg.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    if (p->multi || p->frame) {
      CUDA_TRY(cudaMalloc(&p->d_tile_side, tside.size() * sizeof(uint32_t)));
      CUDA_TRY(cudaMemcpy(p->d_tile_side, tside.data(), tside.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
  }
  p->n_ranges = n_ranges;
  p->n_tiles = (int)tiles.size();
  p->has_blocks = true;
  return ADJ_OK;
}

namespace {

// Chunks of the host-buffer path, their tile lists, streams and events.
int build_host_chunks(adj_plan* p) {
  free_chunks(p);
  const size_t n = p->blocks.size();
  const int64_t full = std::max<int64_t>(kHostChunkCoefs, (p->total + kMaxHostChunks - 1) / kMaxHostChunks);
  int64_t left = 0;
  for (const adj_block_t& b : p->blocks) left += (int64_t)b.w * b.h;
  TileSet ts;
  for (size_t i = 0; i < n;) {
    // chunks ramp up (1/4, 1/2, 1 of the full size) and down again near the end, so the first
    // input copy and the last output copy, which nothing overlaps, stay short
    const int64_t ramp = full >> std::max(0, 2 - (int)p->chunks.size());
    const int64_t target = std::max<int64_t>(full / 4, std::min({full, ramp, left / 2}));
    size_t j = i;
    int64_t coefs = 0;
    while (j < n && (j == i || coefs < target)) {
      coefs += (int64_t)p->blocks[j].w * p->blocks[j].h;
      ++j;
    }
    HostChunk c{};
    c.begin = p->blocks[i].offset;
    c.end = p->blocks[j - 1].offset + (int64_t)p->blocks[j - 1].w * p->blocks[j - 1].h;
    c.tile0 = (int)ts.tiles.size();
    c.r0 = (int)ts.rbeg.size();
    build_tiles(p, i, j, &ts);
    c.n_tiles = (int)ts.tiles.size() - c.tile0;
    c.n_ranges = ts.n_ranges;
    p->chunks.push_back(c);
    left -= coefs;
    i = j;
  }
  if (!ts.tiles.empty()) {
    CUDA_TRY(cudaMalloc(&p->d_ctiles, ts.tiles.size() * sizeof(TileDev)));
    CUDA_TRY(cudaMalloc(&p->d_ctile_blk, ts.tblk.size() * sizeof(uint32_t)));
    CUDA_TRY(cudaMalloc(&p->d_crange, ts.rbeg.size() * sizeof(unsigned)));
    CUDA_TRY(cudaMemcpy(p->d_ctiles, ts.tiles.data(), ts.tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->d_ctile_blk, ts.tblk.data(), ts.tblk.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(p->d_crange, ts.rbeg.data(), ts.rbeg.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
  }
  if (!p->s_in) CUDA_TRY(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
  if (!p->s_out) CUDA_TRY(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
  if (!p->ev_start) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming));
  if (!p->ev_done) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming));
  while (p->ev_in.size() < p->chunks.size()) {
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    p->ev_in.push_back(a);
    CUDA_TRY(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    p->ev_k.push_back(b);
  }
  p->chunks_valid = true;
  return ADJ_OK;
}

// Host buffers: per chunk, input copy on s_in -> kernel on `stream` -> output copy on
// s_out; the call returns when the last output copy has finished.
int run_host(adj_plan* p, bool inverse, const void* h_in, float* h_out, cudaStream_t stream) {
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  if (!h_in || !h_out) return fail(ADJ_ERR_INVALID_ARG, "null host buffer");
  int rc = ensure_host_staging(p);
  if (rc) return rc;
  if (!p->chunks_valid && (rc = build_host_chunks(p))) return rc;
  const size_t in_es = inverse ? 4 : 2;
  const unsigned char* hin = static_cast<const unsigned char*>(h_in);
  unsigned char* din = static_cast<unsigned char*>(p->d_host_in);
  CUDA_TRY(cudaEventRecord(p->ev_start, stream));
  CUDA_TRY(cudaStreamWaitEvent(p->s_in, p->ev_start, 0));
  CUDA_TRY(cudaStreamWaitEvent(p->s_out, p->ev_start, 0));
  for (size_t c = 0; c < p->chunks.size(); ++c) {
    const HostChunk& ch = p->chunks[c];
    const size_t n = (size_t)(ch.end - ch.begin);
    CUDA_TRY(cudaMemcpyAsync(din + ch.begin * in_es, hin + ch.begin * in_es, n * in_es, cudaMemcpyHostToDevice, p->s_in));
    CUDA_TRY(cudaEventRecord(p->ev_in[c], p->s_in));
    CUDA_TRY(cudaStreamWaitEvent(stream, p->ev_in[c], 0));
    if (ch.n_tiles > 0) {
      FusedArgs a{};
      a.tiles = p->d_ctiles + ch.tile0;
      a.tile_blk = p->d_ctile_blk;
      a.tfs = p->d_tfs;
      a.params = p->d_params;
      a.in = p->d_host_in;
      a.out = p->d_host_out;
      a.sched = p->d_sched + (inverse ? 1 : 0);
      a.range_begin = p->d_crange + ch.r0;
      a.n_tiles = ch.n_tiles;
      a.n_ranges = ch.n_ranges;
      const cudaError_t e = launch_fused(inverse, p->threads, inverse ? p->grid_inv : p->grid_fwd, a, stream);
      if (e != cudaSuccess) return cuda_fail(e, "chunk launch");
    }
    CUDA_TRY(cudaEventRecord(p->ev_k[c], stream));
    CUDA_TRY(cudaStreamWaitEvent(p->s_out, p->ev_k[c], 0));
    CUDA_TRY(cudaMemcpyAsync(h_out + ch.begin, p->d_host_out + ch.begin, n * 4, cudaMemcpyDeviceToHost, p->s_out));
  }
  CUDA_TRY(cudaEventRecord(p->ev_done, p->s_out));
  CUDA_TRY(cudaStreamWaitEvent(stream, p->ev_done, 0));
  CUDA_TRY(cudaStreamSynchronize(stream));
  return ADJ_OK;
}


}  // namespace

// Validates a block list against the plan's transforms (sizes, transform indices, alignment,
// bounds, no overlap) and stores it sorted by offset (p->blocks, p->orig).  Host only.
static int accept_blocks(adj_plan* p, const adj_block_t* blocks, int64_t n_blocks, int64_t total_coefs) {
  if (n_blocks < 0 || (n_blocks > 0 && !blocks)) return fail(ADJ_ERR_INVALID_ARG, "bad block list");
  if (total_coefs < 0 || total_coefs > (int64_t(1) << 36)) return fail(ADJ_ERR_INVALID_ARG, "total_coefs %lld out of range", (long long)total_coefs);
  // disjoint blocks of at least 16 samples: no more than total_coefs / 16 of them (which also
  // keeps every block index within the 32-bit tile lists)
  if (n_blocks > total_coefs / 16)
    return fail(ADJ_ERR_INVALID_ARG, "%lld blocks cannot fit in %lld coefficients", (long long)n_blocks, (long long)total_coefs);
  const int n_tfs = (int)p->tfs.size();
  for (int64_t i = 0; i < n_blocks; ++i) {
    const adj_block_t& b = blocks[i];
    if (!is_size(b.w) || !is_size(b.h)) return fail(ADJ_ERR_UNSUPPORTED_SIZE, "block %lld: %dx%d", (long long)i, b.w, b.h);
    if (b.tf_h >= n_tfs || b.tf_v >= n_tfs) return fail(ADJ_ERR_INVALID_ARG, "block %lld: transform index out of range", (long long)i);
    if (p->tfs[b.tf_h].n != b.w || p->tfs[b.tf_v].n != b.h)
      return fail(ADJ_ERR_PARAM_MISMATCH, "block %lld: %dx%d with transforms of length %d (h) and %d (v)",
                  (long long)i, b.w, b.h, p->tfs[b.tf_h].n, p->tfs[b.tf_v].n);
    if (b.offset < 0 || b.offset % 16) return fail(ADJ_ERR_MISALIGNED, "block %lld: offset %lld", (long long)i, (long long)b.offset);
    if (b.offset > total_coefs - (int64_t)b.w * b.h) return fail(ADJ_ERR_INVALID_ARG, "block %lld extends past total_coefs", (long long)i);
  }
  std::vector<int64_t> order(n_blocks);
  for (int64_t i = 0; i < n_blocks; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return blocks[a].offset < blocks[b].offset; });
  for (int64_t i = 1; i < n_blocks; ++i) {
    const adj_block_t &a = blocks[order[i - 1]], &b = blocks[order[i]];
    if (a.offset + (int64_t)a.w * a.h > b.offset) return fail(ADJ_ERR_INVALID_ARG, "blocks %lld and %lld overlap", (long long)order[i - 1], (long long)order[i]);
  }
  p->blocks.clear();
  p->blocks.reserve(n_blocks);
  for (int64_t i : order) p->blocks.push_back(blocks[i]);
  p->orig = order;
  return ADJ_OK;
}

extern "C" {

const char* adj_last_error(void) { return g_err; }

struct adj_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int adj_graph_create(adj_plan_t* p, int32_t what, const void* d_in, float* d_out, float* d_out2, adj_graph_t** graph) try {
  clear_error();
  if (!graph) return fail(ADJ_ERR_INVALID_ARG, "null graph pointer");
  *graph = nullptr;
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (what < ADJ_GRAPH_FWD || what > ADJ_GRAPH_FWD_MULTIPLE) return fail(ADJ_ERR_INVALID_ARG, "unknown graph kind %d", what);
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(d_in, "input")) || (rc = check_ptr(d_out, "output"))) return rc;
  if (what == ADJ_GRAPH_ROUNDTRIP && (rc = check_ptr(d_out2, "second output"))) return rc;
  cudaStream_t s = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(s);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  switch (what) {
    case ADJ_GRAPH_FWD: rc = run(p, false, d_in, d_out, s); break;
    case ADJ_GRAPH_INV: rc = run(p, true, d_in, d_out, s); break;
    case ADJ_GRAPH_FWD_PLAIN: rc = run_plain(p, false, d_in, d_out, s); break;
    case ADJ_GRAPH_INV_PLAIN: rc = run_plain(p, true, d_in, d_out, s); break;
    case ADJ_GRAPH_FWD_MULTIPLE: rc = run_multi(p, static_cast<const int16_t*>(d_in), d_out, d_out2, s); break;
    default:
      rc = run(p, false, d_in, d_out, s);
      if (!rc) rc = run(p, true, d_out, d_out2, s);
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  cudaStreamDestroy(s);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  adj_graph* out = new (std::nothrow) adj_graph();
  if (!out) {
    cudaGraphDestroy(g);
    return fail(ADJ_ERR_NO_MEMORY, "host memory allocation failed");
  }
  out->graph = g;
  e = cudaGraphInstantiate(&out->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete out;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  *graph = out;
  return ADJ_OK;
} catch (...) {
  return entry_exception();
}

int adj_graph_launch(adj_graph_t* g, void* stream) {
  clear_error();
  if (!g) return fail(ADJ_ERR_INVALID_ARG, "null graph");
  CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return ADJ_OK;
}

void adj_graph_destroy(adj_graph_t* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

}  // extern "C"

// Lets other translation units of the library report errors through adj_last_error().
void adjtx::set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

extern "C" {

int adj_plan_create(adj_plan_t** plan, const adj_1d_desc_t* tfs, int32_t n_tfs, int32_t flags) try {
  clear_error();
  if (!plan) return fail(ADJ_ERR_INVALID_ARG, "null plan pointer");
  *plan = nullptr;
  if (n_tfs < 0 || n_tfs > 65535 || (n_tfs > 0 && !tfs)) return fail(ADJ_ERR_INVALID_ARG, "bad transform table (n_tfs=%d)", n_tfs);
  if (flags != ADJ_PLAN_DEFAULT) return fail(ADJ_ERR_INVALID_ARG, "unknown flags %d", flags);
  std::vector<TfHost> hs(n_tfs);
  for (int i = 0; i < n_tfs; ++i) {
    int rc = validate_tf(tfs[i], i, &hs[i]);
    if (rc) return rc;
  }
  // the plan is handed out only complete: an error or exception on the way frees it
  std::unique_ptr<adj_plan, void (*)(adj_plan_t*)> owner(new adj_plan(), adj_plan_destroy);
  adj_plan* p = owner.get();
  p->tfs = std::move(hs);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  int rc = upload_params(p, p->tfs);
  // gradient layouts: accumulator side^2 per transform (band n, post / dense kt) and the
  // gradient entries (band: angles, post: K x K, dense: n x n)
  for (const TfHost& t : p->tfs) {
    const int side = t.kind == ADJ_ADJ_PRE_BAND ? t.n : (t.kind >= ADJ_ADJ_POST_BLOCK ? t.kt : 0);
    const int ng = t.kind == ADJ_ADJ_PRE_BAND ? t.n_pairs : (t.kind >= ADJ_ADJ_POST_BLOCK ? t.k * t.k : 0);
    p->m_off.push_back(p->P);
    p->g_off.push_back(p->n_grad);
    p->kq.push_back(t.k);
    p->P += side * side;
    p->n_grad += ng;
  }
  p->g_off.push_back(p->n_grad);
  if (!rc && !p->tfs.empty()) {
    std::vector<int> lay(p->m_off);
    lay.insert(lay.end(), p->g_off.begin(), p->g_off.end() - 1);
    lay.insert(lay.end(), p->kq.begin(), p->kq.end());
    e = cudaMalloc(&p->d_layout, lay.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_layout, lay.data(), lay.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "gradient layout upload");
  }
  if (!rc) {
    e = cudaMalloc(&p->d_sched, 3 * sizeof(SchedState));
    if (e == cudaSuccess) e = cudaMemset(p->d_sched, 0, 3 * sizeof(SchedState));
    if (e != cudaSuccess) rc = cuda_fail(e, "scheduler state allocation");
  }
  for (int inv = 0; inv < 2 && !rc; ++inv) {
    const void* fn = fused_kernel_ptr(inv, p->threads);
    const int smem = fused_dyn_smem(inv, kModePacked);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p->threads, smem);
    if (e != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    else (inv ? p->occ_inv : p->occ_fwd) = std::max(1, occ);
  }
  if (!rc) {
    const void* fn = multi_kernel_ptr();
    const int smem = fused_dyn_smem(false, kModeMulti);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p->threads, smem);
    if (e != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    else p->occ_multi = std::max(1, occ);
  }
  if (!rc) {
    const void* fn = fwd_f32_kernel_ptr();
    const int smem = fused_dyn_smem(false, kModePackedF32);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p->threads, smem);
    if (e != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    else p->occ_f32 = std::max(1, occ);
  }
  for (int v = 0; v < 3 && !rc; ++v) {  // frame forward, inverse FP32, inverse int16
    const void* fn = frame_kernel_ptr(v > 0, v == 2);
    const int smem = fused_dyn_smem(v > 0, v == 2 ? kModeFrameI16 : kModeFrame);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p->threads, smem);
    if (e != cudaSuccess) rc = cuda_fail(e, "kernel attributes");
    else if (v == 0) p->occ_frame_fwd = std::max(1, occ);
    else p->occ_frame = v == 1 ? std::max(1, occ) : std::min(p->occ_frame, std::max(1, occ));
  }
  if (!rc) {
    for (int i = 0; i < 25; ++i) p->tuning.cap_div[i] = 1;
    p->tuning.ctas_per_sm = 0;
    p->tuning.ranges_per_sm = 1;
    p->tuning.tail_pct = kDefaultTailPct;
    apply_grid(p);
  }
  if (rc) return rc;
  *plan = owner.release();
  return ADJ_OK;
} catch (...) {
  return entry_exception();
}

int adj_plan_update_params(adj_plan_t* p, const adj_1d_desc_t* tfs, int32_t n_tfs) try {
  clear_error();
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (n_tfs != (int)p->tfs.size() || (n_tfs > 0 && !tfs))
    return fail(ADJ_ERR_PARAM_MISMATCH, "update with %d transforms, plan has %zu", n_tfs, p->tfs.size());
  std::vector<TfHost> hs(n_tfs);
  for (int i = 0; i < n_tfs; ++i) {
    int rc = validate_tf(tfs[i], i, &hs[i]);
    if (rc) return rc;
    const TfHost &a = hs[i], &b = p->tfs[i];
    if (a.n != b.n || a.core != b.core || a.kind != b.kind || a.n_layers != b.n_layers || a.parity != b.parity || a.k != b.k)
      return fail(ADJ_ERR_PARAM_MISMATCH, "tf %d: structure changed", i);
  }
  const int rc = upload_params(p, hs);
  if (!rc) p->tfs.swap(hs);
  return rc;
} catch (...) {
  return entry_exception();
}

int adj_plan_set_blocks(adj_plan_t* p, const adj_block_t* blocks, int64_t n_blocks, int64_t total_coefs) try {
  clear_error();
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  int rc = accept_blocks(p, blocks, n_blocks, total_coefs);
  if (rc) return rc;
  p->multi = false;
  p->side_off.clear();
  p->frame = false;
  p->frame_off.clear();
  p->n_blocks = n_blocks;
  p->total = total_coefs;
  rc = build_layout(p);
  if (rc) return rc;
  p->has_blocks = true;
  return ADJ_OK;
} catch (...) {
  if (p) free_blocks(p);
  return entry_exception();
}

int adj_layout_preview(const adj_1d_desc_t* tfs, int32_t n_tfs, const adj_block_t* blocks, int64_t n_blocks,
                       int64_t total_coefs, int32_t n_sm, adj_tile_info_t* tiles, double* costs, int64_t tiles_cap,
                       int64_t* n_tiles, uint32_t* list, int64_t list_cap, int64_t* list_len, uint32_t* range_begin,
                       int32_t ranges_cap, int32_t* n_ranges) try {
  clear_error();
  if (!tfs || n_tfs <= 0 || n_tfs > 65535) return fail(ADJ_ERR_INVALID_ARG, "bad transform table");
  if (n_sm < 1 || n_sm > kMaxRanges) return fail(ADJ_ERR_INVALID_ARG, "n_sm %d out of range", n_sm);
  if (!n_tiles || !list_len || !n_ranges) return fail(ADJ_ERR_INVALID_ARG, "null count pointer");
  adj_plan pl;
  pl.tfs.resize(n_tfs);
  int rc;
  for (int i = 0; i < n_tfs; ++i)
    if ((rc = validate_tf(tfs[i], i, &pl.tfs[i]))) return rc;
  if ((rc = accept_blocks(&pl, blocks, n_blocks, total_coefs))) return rc;
  for (int i = 0; i < 25; ++i) pl.tuning.cap_div[i] = 1;
  pl.tuning.ctas_per_sm = 0;
  pl.tuning.ranges_per_sm = 1;
  pl.tuning.tail_pct = kDefaultTailPct;
  pl.n_sm = n_sm;
  TileSet ts;
  build_tiles(&pl, 0, pl.blocks.size(), &ts);
  *n_tiles = (int64_t)ts.tiles.size();
  *list_len = (int64_t)ts.tblk.size();
  *n_ranges = ts.n_ranges;
  if ((tiles || costs) && tiles_cap < *n_tiles) return fail(ADJ_ERR_INVALID_ARG, "tile arrays hold %lld, need %lld", (long long)tiles_cap, (long long)*n_tiles);
  if (list && list_cap < *list_len) return fail(ADJ_ERR_INVALID_ARG, "list holds %lld, needs %lld", (long long)list_cap, (long long)*list_len);
  if (range_begin && ranges_cap < ts.n_ranges) return fail(ADJ_ERR_INVALID_ARG, "range array holds %d + 1, needs %d + 1", ranges_cap, ts.n_ranges);
  static_assert(sizeof(adj_tile_info_t) == sizeof(TileDev), "tile record layout");
  for (size_t t = 0; t < ts.tiles.size(); ++t) {
    const TileDev& d = ts.tiles[t];
    if (tiles) tiles[t] = adj_tile_info_t{d.blk_begin, d.nblk, d.w, d.h, d.tf_h, d.tf_v, 0};
    if (costs) costs[t] = tile_cost(&pl, d);
  }
  if (list && !ts.tblk.empty()) std::memcpy(list, ts.tblk.data(), ts.tblk.size() * sizeof(uint32_t));
  if (range_begin && !ts.rbeg.empty()) std::memcpy(range_begin, ts.rbeg.data(), ts.rbeg.size() * sizeof(uint32_t));
  return ADJ_OK;
} catch (...) {
  return entry_exception();
}

int adj_transform_fwd(adj_plan_t* p, const int16_t* d_resid, float* d_coef, void* stream) {
  clear_error();
  return run(p, false, d_resid, d_coef, static_cast<cudaStream_t>(stream));
}

int adj_transform_fwd_f32(adj_plan_t* p, const float* d_x, float* d_coef, void* stream) {
  clear_error();
  return run_fwd_f32(p, d_x, d_coef, static_cast<cudaStream_t>(stream));
}

int adj_transform_inv(adj_plan_t* p, const float* d_coef, float* d_resid_out, void* stream) {
  clear_error();
  return run(p, true, d_coef, d_resid_out, static_cast<cudaStream_t>(stream));
}

int adj_plan_set_frame_blocks(adj_plan_t* p, const adj_frame_block_t* blocks, int64_t n_blocks, int32_t frame_w,
                              int32_t frame_h, int32_t stride) try {
  clear_error();
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (n_blocks < 0 || (n_blocks > 0 && !blocks)) return fail(ADJ_ERR_INVALID_ARG, "bad block list");
  if (frame_w <= 0 || frame_h <= 0 || frame_w % 4 || frame_h % 4)
    return fail(ADJ_ERR_INVALID_ARG, "frame %dx%d: sides must be positive multiples of 4", frame_w, frame_h);
  if (stride < frame_w || stride % 8) return fail(ADJ_ERR_MISALIGNED, "frame stride %d: must be >= the width and a multiple of 8", stride);
  if ((int64_t)stride * frame_h > (int64_t(1) << 34)) return fail(ADJ_ERR_INVALID_ARG, "frame too large");
  const int n_tfs = (int)p->tfs.size();
  const int gw = frame_w / 4, gh = frame_h / 4;
  // disjoint blocks cover at least one 4 x 4 cell each
  if (n_blocks > (int64_t)gw * gh)
    return fail(ADJ_ERR_INVALID_ARG, "%lld blocks cannot fit in a %dx%d frame", (long long)n_blocks, frame_w, frame_h);
  std::vector<uint8_t> cover((size_t)gw * gh, 0);  // 4 x 4 cells already taken
  std::vector<adj_block_t> packed(n_blocks);
  std::vector<int64_t> foff(n_blocks);
  int64_t total = 0;
  for (int64_t i = 0; i < n_blocks; ++i) {
    const adj_frame_block_t& b = blocks[i];
    if (!is_size(b.w) || !is_size(b.h)) return fail(ADJ_ERR_UNSUPPORTED_SIZE, "block %lld: %dx%d", (long long)i, b.w, b.h);
    if (b.tf_h >= n_tfs || b.tf_v >= n_tfs) return fail(ADJ_ERR_INVALID_ARG, "block %lld: transform index out of range", (long long)i);
    if (p->tfs[b.tf_h].n != b.w || p->tfs[b.tf_v].n != b.h)
      return fail(ADJ_ERR_PARAM_MISMATCH, "block %lld: %dx%d with transforms of length %d (h) and %d (v)", (long long)i, b.w,
                  b.h, p->tfs[b.tf_h].n, p->tfs[b.tf_v].n);
    if (b.x < 0 || b.y < 0 || b.x % 4 || b.y % 4)
      return fail(ADJ_ERR_MISALIGNED, "block %lld at (%d, %d): positions must be non-negative multiples of 4", (long long)i, b.x, b.y);
    if ((int64_t)b.x + b.w > frame_w || (int64_t)b.y + b.h > frame_h)
      return fail(ADJ_ERR_INVALID_ARG, "block %lld at (%d, %d) leaves the %dx%d frame", (long long)i, b.x, b.y, frame_w, frame_h);
    for (int cy = b.y / 4; cy < (b.y + b.h) / 4; ++cy)
      for (int cx = b.x / 4; cx < (b.x + b.w) / 4; ++cx) {
        uint8_t& c = cover[(size_t)cy * gw + cx];
        if (c) return fail(ADJ_ERR_INVALID_ARG, "block %lld overlaps an earlier block", (long long)i);
        c = 1;
      }
    packed[i] = adj_block_t{total, b.w, b.h, b.tf_h, b.tf_v};
    foff[i] = (int64_t)b.y * stride + b.x;
    total += (int64_t)b.w * b.h;
  }
  // the packed list is in storage order already (offsets increase with the list index)
  p->blocks = packed;
  p->orig.resize(n_blocks);
  for (int64_t i = 0; i < n_blocks; ++i) p->orig[i] = i;
  p->n_blocks = n_blocks;
  p->total = total;
  p->multi = false;
  p->side_off.clear();
  p->frame = true;
  p->frame_w = frame_w;
  p->frame_h = frame_h;
  p->frame_stride = stride;
  p->frame_off = foff;
  const int rc = build_layout(p);
  if (rc) return rc;
  p->has_blocks = true;
  return ADJ_OK;
} catch (...) {
  if (p) free_blocks(p);
  return entry_exception();
}

int adj_transform_fwd_frame(adj_plan_t* p, const int16_t* d_frame, float* d_coef, void* stream) {
  clear_error();
  return run_frame(p, false, d_frame, d_coef, false, static_cast<cudaStream_t>(stream));
}

int adj_transform_inv_frame(adj_plan_t* p, const float* d_coef, float* d_frame_f32, int16_t* d_frame_i16,
                            void* stream) {
  clear_error();
  if (!!d_frame_f32 == !!d_frame_i16) return fail(ADJ_ERR_INVALID_ARG, "give exactly one of the FP32 and int16 outputs");
  if (d_frame_f32) return run_frame(p, true, d_coef, d_frame_f32, false, static_cast<cudaStream_t>(stream));
  return run_frame(p, true, d_coef, d_frame_i16, true, static_cast<cudaStream_t>(stream));
}

int adj_plan_prepare_multiple(adj_plan_t* p, int64_t* side_offsets, int64_t* side_total) try {
  clear_error();
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  if (p->frame) return fail(ADJ_ERR_INVALID_ARG, "the Multiple forward takes a packed block list, not frame blocks");
  auto k_of = [&](int t) { return p->tfs[t].kind == ADJ_ADJ_POST_BLOCK ? p->tfs[t].k : 0; };
  std::vector<int64_t> size(p->blocks.size());
  for (size_t s = 0; s < p->blocks.size(); ++s) {
    const adj_block_t& b = p->blocks[s];
    for (int t : {(int)b.tf_h, (int)b.tf_v}) {
      const TfHost& tf = p->tfs[t];
      if (tf.core != ADJ_CORE_DCT2 || (tf.kind != ADJ_ADJ_NONE && tf.kind != ADJ_ADJ_POST_BLOCK))
        return fail(ADJ_ERR_INVALID_ARG, "block %lld: transform %d is not a DCT-2 with no adjustment or a post-adjustment",
                    (long long)p->orig[s], t);
      if (2 * k_of(t) > tf.n)
        return fail(ADJ_ERR_UNSUPPORTED_SIZE, "block %lld: transform %d has K=%d > n/2", (long long)p->orig[s], t, tf.k);
    }
    const int64_t kh = k_of(b.tf_h), kv = k_of(b.tf_v);
    size[p->orig[s]] = (2 * kv * b.w + 2 * b.h * kh + 3) / 4 * 4;
  }
  std::vector<int64_t> off(p->blocks.size() + 1, 0);
  for (size_t i = 0; i < size.size(); ++i) off[i + 1] = off[i] + size[i];
  if (off.back() / 4 > (int64_t)UINT32_MAX) return fail(ADJ_ERR_INVALID_ARG, "side buffer of %lld floats is too large", (long long)off.back());
  const bool was = p->multi;
  std::vector<int64_t> old;
  old.swap(p->side_off);
  p->side_off = off;
  p->multi = true;
  const int rc = build_layout(p);
  if (rc) {
    p->multi = was;
    p->side_off.swap(old);
    return rc;
  }
  if (side_offsets) std::copy(off.begin(), off.end(), side_offsets);
  if (side_total) *side_total = off.back();
  return ADJ_OK;
} catch (...) {
  if (p) free_blocks(p);
  return entry_exception();
}

int adj_transform_fwd_multiple(adj_plan_t* p, const int16_t* d_resid, float* d_coef, float* d_side, void* stream) {
  clear_error();
  return run_multi(p, d_resid, d_coef, d_side, static_cast<cudaStream_t>(stream));
}

int adj_transform_bwd(adj_plan_t* p, const void* d_x, int32_t x_dtype, const float* d_gy, float* d_gx,
                      float* d_gparams, void* stream) {
  clear_error();
  if (x_dtype != ADJ_DTYPE_INT16 && x_dtype != ADJ_DTYPE_FP32) return fail(ADJ_ERR_INVALID_ARG, "x_dtype %d", x_dtype);
  return run_bwd(p, d_x, x_dtype == ADJ_DTYPE_FP32, d_gy, d_gx, d_gparams, static_cast<cudaStream_t>(stream));
}

int adj_plan_param_layout(const adj_plan_t* p, int32_t* offsets) {
  clear_error();
  if (!p || !offsets) return fail(ADJ_ERR_INVALID_ARG, "null argument");
  for (size_t i = 0; i < p->g_off.size(); ++i) offsets[i] = p->g_off[i];
  return ADJ_OK;
}

int adj_transform_fwd_plain(adj_plan_t* p, const int16_t* d_resid, float* d_coef, void* stream) {
  clear_error();
  return run_plain(p, false, d_resid, d_coef, static_cast<cudaStream_t>(stream));
}

int adj_transform_inv_plain(adj_plan_t* p, const float* d_coef, float* d_resid_out, void* stream) {
  clear_error();
  return run_plain(p, true, d_coef, d_resid_out, static_cast<cudaStream_t>(stream));
}

int adj_transform_fwd_host(adj_plan_t* p, const int16_t* h_resid, float* h_coef, void* stream) try {
  clear_error();
  return run_host(p, false, h_resid, h_coef, static_cast<cudaStream_t>(stream));
} catch (...) {
  return entry_exception();
}

int adj_transform_inv_host(adj_plan_t* p, const float* h_coef, float* h_resid_out, void* stream) try {
  clear_error();
  return run_host(p, true, h_coef, h_resid_out, static_cast<cudaStream_t>(stream));
} catch (...) {
  return entry_exception();
}

int adj_plan_get_tuning(const adj_plan_t* p, adj_tuning_t* t) {
  clear_error();
  if (!p || !t) return fail(ADJ_ERR_INVALID_ARG, "null argument");
  *t = p->tuning;
  return ADJ_OK;
}

int adj_plan_set_tuning(adj_plan_t* p, const adj_tuning_t* t) try {
  clear_error();
  if (!p || !t) return fail(ADJ_ERR_INVALID_ARG, "null argument");
  for (int i = 0; i < 25; ++i)
    if (t->cap_div[i] != 1 && t->cap_div[i] != 2 && t->cap_div[i] != 4 && t->cap_div[i] != 8)
      return fail(ADJ_ERR_INVALID_ARG, "cap_div[%d] = %d", i, t->cap_div[i]);
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > 64) return fail(ADJ_ERR_INVALID_ARG, "ctas_per_sm %d", t->ctas_per_sm);
  if (t->ranges_per_sm < 1 || t->ranges_per_sm > 4) return fail(ADJ_ERR_INVALID_ARG, "ranges_per_sm %d", t->ranges_per_sm);
  if (t->tail_pct < 0 || t->tail_pct > 50) return fail(ADJ_ERR_INVALID_ARG, "tail_pct %d", t->tail_pct);
  p->tuning = *t;
  apply_grid(p);
  if (p->has_blocks) return build_layout(p);
  return ADJ_OK;
} catch (...) {
  if (p) free_blocks(p);
  return entry_exception();
}

namespace {

// FNV-1a over the block-size / transform-kind histogram: the workload signature of a tuning.
uint64_t signature(const adj_plan* p) {
  std::vector<uint64_t> hist(25 * 16, 0);
  for (const adj_block_t& b : p->blocks) {
    const int cls = (ilog2(b.w) - 2) * 5 + (ilog2(b.h) - 2);
    hist[cls * 16 + p->tfs[b.tf_h].kind * 4 + p->tfs[b.tf_v].kind] += 1;
  }
  uint64_t h = 1469598103934665603ull;
  for (uint64_t v : hist) {
    // quantise counts to ~3% so that equal workloads of other seeds share a tuning
    uint64_t q = v;
    while (q >= 64) q >>= 1;  // keep the top bits
    uint64_t lg = 0;
    for (uint64_t t = v; t >= 64; t >>= 1) ++lg;
    const uint64_t key = (lg << 8) | q;
    for (int i = 0; i < 8; ++i) {
      h ^= (key >> (8 * i)) & 0xff;
      h *= 1099511628211ull;
    }
  }
  return h;
}

std::string device_name(int dev) {
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string s = prop.name;
  for (char& c : s)
    if (c == ' ' || c == '"') c = '_';
  return s;
}

// Cache lines: "<device> <signature hex> <ctas> <ranges> <tail_pct> <25 cap_div>"
bool cache_lookup(const char* path, const std::string& dev, uint64_t sig, adj_tuning_t* t) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char name[256];
  unsigned long long s;
  adj_tuning_t c{};
  bool found = false;
  while (fscanf(f, "%255s %llx %d %d %d", name, &s, &c.ctas_per_sm, &c.ranges_per_sm, &c.tail_pct) == 5) {
    bool ok = true;
    for (int i = 0; i < 25 && ok; ++i) ok = fscanf(f, "%d", &c.cap_div[i]) == 1;
    if (!ok) break;
    if (dev == name && s == sig) {
      *t = c;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& dev, uint64_t sig, const adj_tuning_t& t) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %llx %d %d %d", dev.c_str(), (unsigned long long)sig, t.ctas_per_sm, t.ranges_per_sm, t.tail_pct);
  for (int i = 0; i < 25; ++i) fprintf(f, " %d", t.cap_div[i]);
  fprintf(f, "\n");
  fclose(f);
}

// median forward + inverse time (ms) of the plan as tuned now
int time_plan(adj_plan* p, const int16_t* x, float* y, float* xr, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best[5];
  int rc = run(p, false, x, y, s);
  if (!rc) rc = run(p, true, y, xr, s);
  for (int r = 0; r < 5 && !rc; ++r) {
    cudaEventRecord(e0, s);
    rc = run(p, false, x, y, s);
    if (!rc) rc = run(p, true, y, xr, s);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
    if (!rc) cudaEventElapsedTime(&best[r], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  std::sort(best, best + 5);
  *ms = best[2];
  return ADJ_OK;
}

}  // namespace

int adj_plan_autotune(adj_plan_t* p, const int16_t* x, float* y, float* xr, const char* cache_path, int32_t max_evals,
                      void* stream_) try {
  clear_error();
  if (!p) return fail(ADJ_ERR_INVALID_ARG, "null plan");
  if (!p->has_blocks) return fail(ADJ_ERR_NO_BLOCKS, "adj_plan_set_blocks has not been called");
  int rc;
  if ((rc = check_ptr(x, "input")) || (rc = check_ptr(y, "coefficients")) || (rc = check_ptr(xr, "reconstruction")))
    return rc;
  if (p->n_tiles == 0) return ADJ_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream_);
  const std::string dev = device_name(p->device);
  const uint64_t sig = signature(p);
  adj_tuning_t t{};
  if (cache_lookup(cache_path, dev, sig, &t)) return adj_plan_set_tuning(p, &t);

  int evals = 0;
  auto budget = [&]() { return max_evals <= 0 || evals < max_evals; };
  adj_tuning_t best = p->tuning;
  float best_ms = 0.f;
  if ((rc = time_plan(p, x, y, xr, s, &best_ms))) return rc;
  auto trial = [&](const adj_tuning_t& cand) -> int {
    if (!budget()) return ADJ_OK;
    ++evals;
    int r = adj_plan_set_tuning(p, &cand);
    float ms = 0.f;
    if (!r) r = time_plan(p, x, y, xr, s, &ms);
    if (r) return r;
    if (ms < best_ms * 0.99f) {
      best_ms = ms;
      best = cand;
    }
    return ADJ_OK;
  };
  // share of the cheapest tiles dealt over the ends of the ranges, then persistent CTAs per
  // SM, then ranges per SM
  for (int tp : {0, 5, 10, 20}) {
    if (tp == best.tail_pct) continue;
    adj_tuning_t cand = best;
    cand.tail_pct = tp;
    if ((rc = trial(cand))) return rc;
  }
  const int occ = std::min(p->occ_fwd, p->occ_inv);
  for (int c = occ - 1; c >= std::max(2, occ - 2); --c) {
    adj_tuning_t cand = best;
    cand.ctas_per_sm = c;
    if ((rc = trial(cand))) return rc;
  }
  for (int r = 2; r <= 4; r *= 2) {
    adj_tuning_t cand = best;
    cand.ranges_per_sm = r;
    if ((rc = trial(cand))) return rc;
  }
  // tile capacity per block size, largest coefficient shares first
  std::vector<std::pair<int64_t, int>> share(25);
  for (int i = 0; i < 25; ++i) share[i] = {0, i};
  for (const adj_block_t& b : p->blocks) share[(ilog2(b.w) - 2) * 5 + (ilog2(b.h) - 2)].first += (int64_t)b.w * b.h;
  std::sort(share.rbegin(), share.rend());
  for (const auto& sc : share) {
    if (sc.first == 0) break;
    const int cls = sc.second;
    const int w = 4 << (cls / 5), h = 4 << (cls % 5);
    for (int div = 2; div <= 8; div *= 2) {
      if (tile_capacity(w, h) / div < 1) break;
      adj_tuning_t cand = best;
      cand.cap_div[cls] = div;
      if ((rc = trial(cand))) return rc;
    }
  }
  if ((rc = adj_plan_set_tuning(p, &best))) return rc;
  cache_store(cache_path, dev, sig, best);
  return ADJ_OK;
} catch (...) {
  if (p) free_blocks(p);
  return entry_exception();
}

int adj_plan_info(const adj_plan_t* p, adj_plan_info_t* info) {
  clear_error();
  if (!p || !info) return fail(ADJ_ERR_INVALID_ARG, "null argument");
  info->n_blocks = p->n_blocks;
  info->total_coefs = p->total;
  info->n_tiles = p->n_tiles;
  info->grid_fwd = p->grid_fwd;
  info->grid_inv = p->grid_inv;
  info->threads = p->threads;
  info->smem_bytes = kSmemBytes;
  info->n_sm = p->n_sm;
  return ADJ_OK;
}

void adj_plan_destroy(adj_plan_t* p) {
  if (!p) return;
  free_blocks(p);
  for (cudaEvent_t e : p->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_k) cudaEventDestroy(e);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_done) cudaEventDestroy(p->ev_done);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  cudaFree(p->d_tfs);
  cudaFree(p->d_params);
  cudaFree(p->d_sched);
  cudaFree(p->d_host_in);
  cudaFree(p->d_host_out);
  cudaFree(p->d_layout);
  cudaFree(p->d_partial);
  cudaFree(p->d_M);
  delete p;
}

}  // extern "C"
