// Forward transform of a uniform batch without any device allocation.
//
// Some callers cannot allocate device memory on their processing path: a real-time
// encoder that reserves all of its GPU memory at start-up and must not call
// cudaMalloc/cudaFree per frame (those calls can synchronise the device and stall the
// other streams of the pipeline), or a plug-in running inside a host framework that
// owns the device memory and gives plug-ins no allocator.  For them,
// adj_transform_fwd_uniform_noalloc runs the same fused forward kernel as
// adj_transform_fwd, but everything the kernel needs beside its input and output (work
// counter, transform records, FP32 parameters, tile list and block offsets) lives in
// one file-scope static device array, g_noalloc_scratch, instead of plan memory.
//
// The array is ADJ_NOALLOC_SCRATCH_BYTES (3 MiB) on every device that loads the library,
// held until the process exits.  Its device address is taken once per device with
// cudaGetSymbolAddress, on the first call made while that device is current.  All calls
// share the array and it keeps the previous call's contents; each call clears the work
// scheduling state and rewrites everything else it reads.  Calls that overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by the caller.
//
// The records and parameters are uploaded from host memory that lives only for the call (the
// caller's stack and a per-thread array reused by the next call).  A copy recorded into a
// CUDA graph would read that memory again at every replay, long after it is gone, so a call
// made while its stream is capturing is rejected before anything is enqueued.  Because the
// uploads come from pageable memory, the call may also block the host until the work already
// queued on the stream has finished.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "adjtx.h"
#include "adjtx_kernels.h"

using namespace adjtx;

namespace {

constexpr size_t kScratchBytes = ADJ_NOALLOC_SCRATCH_BYTES;
constexpr size_t kSchedOff = 0;                                     // SchedState
constexpr size_t kRangeOff = ((sizeof(SchedState) + 255) / 256) * 256;  // {0, n_tiles}
constexpr size_t kTfOff = kRangeOff + 256;                           // 2 TfDev records
constexpr size_t kParamOff = kTfOff + 256;                            // FP32 parameters
// A transform carries a band or a post block, never both.  A band has at most 64 layers x 32
// (cos, sin) pairs, stored twice (back to back, and per layer padded to n / 2 pairs): 8192
// floats; a post block at most 64 x 64 = 4096, stored with its transpose: 8192.  Plus alignment
// padding.
constexpr size_t kMaxParamFloats = 2 * 8200 + 32;
constexpr size_t kTileOff = kParamOff + ((kMaxParamFloats * 4 + 255) / 256) * 256;
constexpr size_t kTileBytes = (size_t)ADJ_NOALLOC_MAX_BLOCKS * sizeof(TileDev);
constexpr size_t kBlkOff = kTileOff + kTileBytes;
constexpr size_t kScratchNeed = kBlkOff + (size_t)ADJ_NOALLOC_MAX_BLOCKS * sizeof(uint32_t);
// (+16: the kernel copies a tile's offsets from the 16-byte aligned address below the
// list and up to 3 entries past it)
static_assert(kScratchNeed + 16 <= kScratchBytes, "scratch layout exceeds the static array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
constexpr int kThreads = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices];
int g_grid[kMaxDevices];

int err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

int cuda_err(cudaError_t e, const char* what) {
  return err(ADJ_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool is_size(int n) { return n == 4 || n == 8 || n == 16 || n == 32 || n == 64; }

// Per-device set-up: device address of the static array and the persistent grid size.
int setup(int dev, unsigned char** ptr, int* grid) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    int n_sm = 0, occ = 0;
    const void* fn = fused_kernel_ptr(false, kThreads);
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int smem = fused_dyn_smem(false, kModePacked);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
    if (e != cudaSuccess) return cuda_err(e, "no-alloc set-up");
    g_grid[dev] = (occ > 0 ? occ : 1) * n_sm;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  *grid = g_grid[dev];
  return ADJ_OK;
}

// Checks one 1-D transform and writes its record and FP32 parameters (cos/sin per angle,
// Q padded to KT x KT with the identity) into host arrays on the caller's stack.
int pack_tf(const adj_1d_desc_t* d, const char* name, TfDev* rec, float* params, size_t* n_params) {
  if (!d) return err(ADJ_ERR_INVALID_ARG, "%s is null", name);
  if (!is_size(d->n)) return err(ADJ_ERR_UNSUPPORTED_SIZE, "%s: n=%d not in {4,8,16,32,64}", name, d->n);
  if (d->core < 0 || d->core > 3) return err(ADJ_ERR_INVALID_ARG, "%s: core %d", name, d->core);
  if (d->kind < 0 || d->kind > 3) return err(ADJ_ERR_INVALID_ARG, "%s: kind %d", name, d->kind);
  if (d->kind == ADJ_ADJ_DENSE && d->k != d->n)
    return err(ADJ_ERR_PARAM_MISMATCH, "%s: a dense transform needs k = n", name);
  std::memset(rec, 0, sizeof *rec);
  rec->n = d->n;
  rec->core = d->core;
  rec->kind = d->kind;
  size_t np = *n_params;
  if (d->kind == ADJ_ADJ_PRE_BAND) {
    if (d->n_layers < 0 || d->n_layers > ADJ_MAX_LAYERS)
      return err(ADJ_ERR_UNSUPPORTED_SIZE, "%s: %d layers (max %d)", name, d->n_layers, ADJ_MAX_LAYERS);
    if (d->n_layers > 0 && !d->layer_parity) return err(ADJ_ERR_INVALID_ARG, "%s: null layer_parity", name);
    int pairs = 0;
    for (int l = 0; l < d->n_layers; ++l) {
      const int par = d->layer_parity[l];
      if (par > 1) return err(ADJ_ERR_INVALID_ARG, "%s: parity of layer %d is %d", name, l, par);
      if (par) {
        if (l < 32) rec->par_lo |= 1u << l;
        else rec->par_hi |= 1u << (l - 32);
      }
      pairs += par ? d->n / 2 - 1 : d->n / 2;
    }
    if (pairs > 0 && !d->angles) return err(ADJ_ERR_INVALID_ARG, "%s: null angles", name);
    rec->n_layers = d->n_layers;
    rec->n_pairs = pairs;
    if (np % 2) params[np++] = 0.f;
    rec->cs_off = (uint32_t)(np / 2);
    for (int i = 0; i < pairs; ++i) {
      if (!std::isfinite(d->angles[i])) return err(ADJ_ERR_PARAM_MISMATCH, "%s: non-finite angle", name);
      params[np++] = (float)std::cos(d->angles[i]);
      params[np++] = (float)std::sin(d->angles[i]);
    }
    // per-layer table of the kernels: n / 2 (cos, sin) pairs a layer, 16-byte aligned
    while (np % 4) params[np++] = 0.f;
    rec->csl_off = (uint32_t)(np / 4);
    for (int l = 0, a = 0; l < d->n_layers; ++l) {
      const int lp = d->layer_parity[l] ? d->n / 2 - 1 : d->n / 2;
      for (int j = 0; j < d->n / 2; ++j) {
        params[np++] = j < lp ? (float)std::cos(d->angles[a + j]) : 1.f;
        params[np++] = j < lp ? (float)std::sin(d->angles[a + j]) : 0.f;
      }
      a += lp;
    }
  } else if (d->kind == ADJ_ADJ_POST_BLOCK || d->kind == ADJ_ADJ_DENSE) {
    const int k = d->k;
    if (k < 1 || k > d->n) return err(ADJ_ERR_UNSUPPORTED_SIZE, "%s: K=%d with n=%d", name, k, d->n);
    rec->k = k;
    if (!d->q) return err(ADJ_ERR_INVALID_ARG, "%s: null q", name);
    double worst = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int r = 0; r < k; ++r) s += d->q[r * k + i] * d->q[r * k + j];
        if (!std::isfinite(s)) return err(ADJ_ERR_PARAM_MISMATCH, "%s: non-finite Q", name);
        worst = std::fmax(worst, std::fabs(s - (i == j ? 1.0 : 0.0)));
      }
    if (worst > 1e-6) return err(ADJ_ERR_PARAM_MISMATCH, "%s: Q not orthogonal (%g)", name, worst);
    int kt = 4;
    while (kt < k) kt *= 2;
    rec->kt = kt;
    while (np % 4) params[np++] = 0.f;
    rec->q_off = (uint32_t)np;
    for (int i = 0; i < kt; ++i)
      for (int j = 0; j < kt; ++j)
        params[np++] = (float)((i < k && j < k) ? d->q[i * k + j] : (i == j ? 1.0 : 0.0));
    rec->qt_off = (uint32_t)np;
    for (int j = 0; j < kt; ++j)
      for (int i = 0; i < kt; ++i)
        params[np++] = (float)((i < k && j < k) ? d->q[i * k + j] : (i == j ? 1.0 : 0.0));
  }
  *n_params = np;
  return ADJ_OK;
}

// Tile list of a uniform batch: tile t holds blocks [t*cap, min((t+1)*cap, n)).
__global__ void noalloc_tiles_kernel(TileDev* tiles, uint32_t* blk, int n_blocks, int n_tiles, int cap,
                                     int w, int h, uint32_t words16) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_blocks; i += gridDim.x * blockDim.x)
    blk[i] = (uint32_t)i * words16;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
    TileDev d{};
    d.blk_begin = (uint32_t)(t * cap);
    const int left = n_blocks - t * cap;
    d.nblk = (uint16_t)(left < cap ? left : cap);
    d.w = (uint16_t)w;
    d.h = (uint16_t)h;
    d.tf_h = 0;
    d.tf_v = 1;
    tiles[t] = d;
  }
}

}  // namespace

extern "C" int adj_transform_fwd_uniform_noalloc(const adj_1d_desc_t* tf_h, const adj_1d_desc_t* tf_v,
                                                 int64_t n_blocks, const int16_t* d_resid, float* d_coef,
                                                 void* stream_) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (n_blocks < 0) return err(ADJ_ERR_INVALID_ARG, "n_blocks %lld < 0", (long long)n_blocks);
  if (n_blocks > ADJ_NOALLOC_MAX_BLOCKS)
    return err(ADJ_ERR_UNSUPPORTED_SIZE, "n_blocks %lld exceeds ADJ_NOALLOC_MAX_BLOCKS (%d)", (long long)n_blocks,
               ADJ_NOALLOC_MAX_BLOCKS);
  if (!d_resid || !d_coef) return err(ADJ_ERR_INVALID_ARG, "null device buffer");
  if (reinterpret_cast<uintptr_t>(d_resid) % 16 || reinterpret_cast<uintptr_t>(d_coef) % 16)
    return err(ADJ_ERR_MISALIGNED, "device buffers must be 16-byte aligned");
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(stream, &capture);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaStreamIsCapturing");
  if (capture != cudaStreamCaptureStatusNone)
    return err(ADJ_ERR_INVALID_ARG,
               "adj_transform_fwd_uniform_noalloc cannot be recorded into a CUDA graph: its uploads read "
               "host memory that lives only for the call");

  TfDev recs[2];
  // per-thread host staging of the parameters (a static array: no allocation per call)
  static thread_local float params[kMaxParamFloats];
  size_t np = 0;
  int rc = pack_tf(tf_h, "tf_h", &recs[0], params, &np);
  if (!rc) rc = pack_tf(tf_v, "tf_v", &recs[1], params, &np);
  if (rc) return rc;
  while (np % 4) params[np++] = 0.f;
  if (n_blocks == 0) return ADJ_OK;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return err(ADJ_ERR_INVALID_ARG, "device %d beyond %d", dev, kMaxDevices);
  unsigned char* base = nullptr;
  int grid = 0;
  rc = setup(dev, &base, &grid);
  if (rc) return rc;

  const int w = recs[0].n, h = recs[1].n;
  const int cap = tile_capacity(w, h);
  const int nb = (int)n_blocks;
  const int n_tiles = (nb + cap - 1) / cap;
  SchedState* sched = reinterpret_cast<SchedState*>(base + kSchedOff);
  TileDev* tiles = reinterpret_cast<TileDev*>(base + kTileOff);
  uint32_t* blk = reinterpret_cast<uint32_t*>(base + kBlkOff);

  unsigned* range_begin = reinterpret_cast<unsigned*>(base + kRangeOff);
  const unsigned ranges[2] = {0u, (unsigned)n_tiles};
  e = cudaMemsetAsync(sched, 0, sizeof(SchedState), stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(range_begin, ranges, sizeof ranges, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kTfOff, recs, sizeof recs, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kParamOff, params, np * sizeof(float), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_err(e, "no-alloc upload");
  const int setup_threads = 256;
  const int setup_grid = (nb + setup_threads - 1) / setup_threads;
  noalloc_tiles_kernel<<<setup_grid < 1024 ? setup_grid : 1024, setup_threads, 0, stream>>>(
      tiles, blk, nb, n_tiles, cap, w, h, (uint32_t)(w * h / 16));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(e, "no-alloc tile set-up launch");

  FusedArgs a{};
  a.tiles = tiles;
  a.tile_blk = blk;
  a.tfs = reinterpret_cast<const TfDev*>(base + kTfOff);
  a.params = reinterpret_cast<const float*>(base + kParamOff);
  a.in = d_resid;
  a.out = d_coef;
  a.sched = sched;
  a.range_begin = range_begin;
  a.n_tiles = n_tiles;
  a.n_ranges = 1;
  e = launch_fused(false, kThreads, grid, a, stream);
  if (e != cudaSuccess) return cuda_err(e, "no-alloc forward launch");
  return ADJ_OK;
}
