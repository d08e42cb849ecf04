// Backward of the adjusted 2-D transforms: gradients with respect to the input and to
// the adjustment parameters, for fitting the adjustments (the paper designs them by a
// non-convex least-squares fit, Eq. 2, with the Givens factorisation after it).
//
// For Y = H_v X H_h^T and G = dL/dY:
//   dL/dX   = H_v^T G H_h                      (the inverse transform of G)
//   dL/dH_h = sum_rows   g~_r x_r^T   with G~ = H_v^T G  (row gradients of U = X H_h^T)
//   dL/dH_v = sum_cols   g_c  u_c^T   with u_c the columns of U
// and for one direction's H = C B A:
//   band  (H = B A):      dL/dA = sum (B^T g) x^T
//   post  (H = C B):      dL/dQ = sum g[:K] (B x)[:K]^T
//   dense (H = D):        dL/dD = sum g x^T
// so every parameter gradient is a sum over lines of outer products a b^T.  The kernel
// forms a and b per line, stages them in shared memory and accumulates M += A^T B with a
// register-tiled FP32 product; each CTA keeps its own partial M per transform (tiles are
// assigned statically), and a fixed-order FP64 reduction and a small finishing kernel (the
// Givens-layer walk for band angles) follow, so results are bit-reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "adjtx_device.cuh"
#include "adjtx_kernels.h"

namespace adjtx {

namespace {

constexpr int kBT = kBwdThreads;
constexpr int kTileF = kTileCoefs;          // floats per tile buffer
// dynamic smem: X/U, G/G~, A, B, M_h, M_v
constexpr int kBwdSmem = 6 * kTileF * 4;

// Size of a transform's outer-product accumulator side (0: no parameters).
__device__ __forceinline__ int m_side(const TfDev& tf) {
  return tf.kind == KIND_BAND ? tf.n : (tf.kind >= KIND_POST ? tf.kt : 0);
}

// Copies one FP32 or int16 block row-major global -> swizzled tile buffer (synchronous,
// cooperative; the backward is not latency-critical enough to double-buffer).
template <bool I16>
__device__ void load_tile(const TileDev& td, const uint32_t* offs, const void* src, float* buf) {
  const int w = td.w, h = td.h, n = td.nblk * w * h;
  for (int e = threadIdx.x; e < n; e += kBT) {
    const int per = w * h;
    const int b = e / per, rem = e - b * per, r = rem / w, c = rem - r * w;
    const size_t g = (size_t)offs[b] * 16 + rem;
    const float v = I16 ? (float)static_cast<const int16_t*>(src)[g] : static_cast<const float*>(src)[g];
    buf[b * per + sw_index(r, c, w)] = v;
  }
}

// M (side n x n, row-major in smem) += A^T B over `lines` lines, A and B swizzled rows of n.
__device__ void accumulate(float* M, const float* As, const float* Bs, int n, int lines) {
  const int nb = n / 4;
  for (int item = threadIdx.x; item < nb * nb; item += kBT) {
    const int bi = item / nb, bj = item - bi * nb;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int l = 0; l < lines; ++l) {
      const int f = sw_f(l, n);
      const float4 a = *reinterpret_cast<const float4*>(As + l * n + ((bi ^ f) << 2));
      const float4 b = *reinterpret_cast<const float4*>(Bs + l * n + ((bj ^ f) << 2));
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float4* m = reinterpret_cast<float4*>(M + (bi * 4 + r) * n + bj * 4);
      float4 o = *m;
      o.x += acc[r][0]; o.y += acc[r][1]; o.z += acc[r][2]; o.w += acc[r][3];
      *m = o;
    }
  }
}

// Stores the first K values of a line as row l of a swizzled K-wide buffer.
template <int K, int N>
__device__ __forceinline__ void stage_vec(float* S, int l, const float (&v)[N]) {
  static_assert(K <= N, "stage width");
  float t[K];
#pragma unroll
  for (int i = 0; i < K; ++i) t[i] = v[i];
  RowSw{S + l * K, sw_f(l, K)}.template store<K>(t);
}

template <int N>
__device__ __forceinline__ void stage_first(float* S, int l, int k, const float (&v)[N]) {
  switch (k) {
    case 4: stage_vec<4, N>(S, l, v); break;
    case 8: if constexpr (N >= 8) stage_vec<8, N>(S, l, v); break;
    case 16: if constexpr (N >= 16) stage_vec<16, N>(S, l, v); break;
    case 32: if constexpr (N >= 32) stage_vec<32, N>(S, l, v); break;
    default: if constexpr (N >= 64) stage_vec<64, N>(S, l, v); break;
  }
}

// Column pass of the backward: per column c of block b, u = U[:, c], g = G[:, c].
// Stages (a, b) of the vertical gradient and replaces G[:, c] by H_v^T g.
template <int H, int W>
__device__ void bwd_col(const TfDev& tf, const float* P, float* bufU, float* bufG, float* As, float* Bs, int nb) {
  constexpr int lgw = ilog2(W);
  const int k = m_side(tf);
  for (int l = threadIdx.x; l < nb * W; l += kBT) {
    const int b = l >> lgw, c = l & (W - 1);
    ColSw<W> colU(bufU + b * W * H, c);
    ColSw<W> colG(bufG + b * W * H, c);
    float g[H], u[H];
    colG.template load<H>(g);
    colU.template load<H>(u);
    if (tf.kind == KIND_BAND) {
      core_apply<H>(tf.core ^ 1, g);           // a = B^T g
      stage_first<H>(As, l, k, g);
      stage_first<H>(Bs, l, k, u);             // b = u
      band<H, true>(g, tf, P);                 // g~ = A^T B^T g
    } else if (tf.kind >= KIND_POST) {
      stage_first<H>(As, l, k, g);             // a = g[:K]
      if (tf.kind == KIND_POST) core_apply<H>(tf.core, u);
      stage_first<H>(Bs, l, k, u);             // b = (B u)[:K]  (dense: u)
      post_inv<H>(g, tf, P, colG);             // C^T g, read back from the column
      if (tf.kind == KIND_POST) core_apply<H>(tf.core ^ 1, g);
    } else {
      core_apply<H>(tf.core ^ 1, g);
    }
    // write g~ back into the column (only this thread touches column c)
    constexpr int SH = sw_shift(W), MK = sw_mask(W);
    float* base = bufG + b * W * H;
#pragma unroll
    for (int i = 0; i < H; ++i) base[i * W + ((((c >> 2) ^ ((i >> SH) & MK))) << 2) + (c & 3)] = g[i];
  }
}

// Row pass of the backward: per row r, u = U[r, :], g~ = G~[r, :].  Stages (a, b) of the
// horizontal gradient and writes dL/dX[r, :] = H_h^T g~ when gx is given.
template <int W>
__device__ void bwd_row(const TfDev& tf, const float* P, const float* bufU, float* bufG, float* As, float* Bs,
                        int nb, int h, const uint32_t* offs, float* gx) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  const int k = m_side(tf);
  const int lgh = lg2(h);
  for (int l = threadIdx.x; l < nb * h; l += kBT) {
    const int b = l >> lgh, r = l & (h - 1);
    RowSw rowU{const_cast<float*>(bufU) + l * W, (r >> SH) & MK};
    RowSw rowG{bufG + l * W, (r >> SH) & MK};
    float g[W], u[W];
    rowG.template load<W>(g);
    rowU.template load<W>(u);
    if (tf.kind == KIND_BAND) {
      core_apply<W>(tf.core ^ 1, g);           // a = B^T g~
      stage_first<W>(As, l, k, g);
      core_apply<W>(tf.core ^ 1, u);           // x = A^T B^T u
      band<W, true>(u, tf, P);
      stage_first<W>(Bs, l, k, u);
      band<W, true>(g, tf, P);                 // dL/dx = A^T B^T g~
    } else if (tf.kind >= KIND_POST) {
      stage_first<W>(As, l, k, g);             // a = g~[:K]
      post_inv<W>(u, tf, P, rowU);             // B x = C^T u  (dense: x = D^T u)
      stage_first<W>(Bs, l, k, u);
      post_inv<W>(g, tf, P, rowG);
      if (tf.kind == KIND_POST) core_apply<W>(tf.core ^ 1, g);
    } else {
      core_apply<W>(tf.core ^ 1, g);
    }
    if (gx) {
      float* dst = gx + (size_t)offs[b] * 16 + r * W;
#pragma unroll
      for (int q = 0; q < W / 4; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
    }
  }
}

// Row pass of the forward on the tile (U = X H_h^T), in place.
template <int W>
__device__ void fwd_row(const TfDev& tf, const float* P, float* buf, int nb, int h) {
  constexpr int SH = sw_shift(W), MK = sw_mask(W);
  for (int l = threadIdx.x; l < nb * h; l += kBT) {
    const int r = l & (h - 1);
    RowSw row{buf + l * W, (r >> SH) & MK};
    line_transform<W, false, false>(tf, P, row, row);
  }
}

template <int H>
__device__ void bwd_col_w(int w, const TfDev& tf, const float* P, float* bufU, float* bufG, float* As, float* Bs,
                          int nb) {
  switch (w) {
    case 4: bwd_col<H, 4>(tf, P, bufU, bufG, As, Bs, nb); break;
    case 8: bwd_col<H, 8>(tf, P, bufU, bufG, As, Bs, nb); break;
    case 16: bwd_col<H, 16>(tf, P, bufU, bufG, As, Bs, nb); break;
    case 32: bwd_col<H, 32>(tf, P, bufU, bufG, As, Bs, nb); break;
    default: bwd_col<H, 64>(tf, P, bufU, bufG, As, Bs, nb); break;
  }
}

// Adds a CTA's accumulator into its own slot of the partial sums and clears it.
__device__ void flush(float* M, int side, float* slot) {
  __syncthreads();
  for (int i = threadIdx.x; i < side * side; i += kBT) {
    slot[i] += M[i];
    M[i] = 0.f;
  }
  __syncthreads();
}

template <bool I16>
__global__ void __launch_bounds__(kBT, 1) bwd_kernel(BwdArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* bufU = sm;
  float* bufG = sm + kTileF;
  float* As = sm + 2 * kTileF;
  float* Bs = sm + 3 * kTileF;
  float* Mh = sm + 4 * kTileF;
  float* Mv = sm + 5 * kTileF;
  __shared__ uint32_t sOff[kMaxTileBlocks];
  float* slot = a.partial + (size_t)blockIdx.x * a.P;
  for (int i = threadIdx.x; i < 2 * kTileF; i += kBT) Mh[i] = 0.f;  // Mh and Mv
  int cur_h = -1, cur_v = -1;  // transforms whose sums Mh / Mv hold
  __syncthreads();

  for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
    const TileDev td = a.tiles[t];
    const TfDev th = a.tfs[td.tf_h], tv = a.tfs[td.tf_v];
    if (cur_h >= 0 && cur_h != td.tf_h) flush(Mh, m_side(a.tfs[cur_h]), slot + a.m_off[cur_h]);
    if (cur_v >= 0 && cur_v != td.tf_v) flush(Mv, m_side(a.tfs[cur_v]), slot + a.m_off[cur_v]);
    cur_h = td.tf_h;
    cur_v = td.tf_v;
    for (int b = threadIdx.x; b < td.nblk; b += kBT) sOff[b] = a.tile_blk[td.blk_begin + b];
    __syncthreads();
    load_tile<I16>(td, sOff, a.x, bufU);
    load_tile<false>(td, sOff, a.gy, bufG);
    __syncthreads();
    const int w = td.w, h = td.h, nb = td.nblk;
    // U = X H_h^T
    switch (w) {
      case 4: fwd_row<4>(th, a.params, bufU, nb, h); break;
      case 8: fwd_row<8>(th, a.params, bufU, nb, h); break;
      case 16: fwd_row<16>(th, a.params, bufU, nb, h); break;
      case 32: fwd_row<32>(th, a.params, bufU, nb, h); break;
      default: fwd_row<64>(th, a.params, bufU, nb, h); break;
    }
    __syncthreads();
    // vertical gradient; G -> G~ = H_v^T G
    switch (h) {
      case 4: bwd_col_w<4>(w, tv, a.params, bufU, bufG, As, Bs, nb); break;
      case 8: bwd_col_w<8>(w, tv, a.params, bufU, bufG, As, Bs, nb); break;
      case 16: bwd_col_w<16>(w, tv, a.params, bufU, bufG, As, Bs, nb); break;
      case 32: bwd_col_w<32>(w, tv, a.params, bufU, bufG, As, Bs, nb); break;
      default: bwd_col_w<64>(w, tv, a.params, bufU, bufG, As, Bs, nb); break;
    }
    __syncthreads();
    if (m_side(tv)) accumulate(Mv, As, Bs, m_side(tv), nb * w);
    __syncthreads();
    // horizontal gradient; dL/dX
    switch (w) {
      case 4: bwd_row<4>(th, a.params, bufU, bufG, As, Bs, nb, h, sOff, a.gx); break;
      case 8: bwd_row<8>(th, a.params, bufU, bufG, As, Bs, nb, h, sOff, a.gx); break;
      case 16: bwd_row<16>(th, a.params, bufU, bufG, As, Bs, nb, h, sOff, a.gx); break;
      case 32: bwd_row<32>(th, a.params, bufU, bufG, As, Bs, nb, h, sOff, a.gx); break;
      default: bwd_row<64>(th, a.params, bufU, bufG, As, Bs, nb, h, sOff, a.gx); break;
    }
    __syncthreads();
    if (m_side(th)) accumulate(Mh, As, Bs, m_side(th), nb * h);
    __syncthreads();
  }
  if (cur_h >= 0) flush(Mh, m_side(a.tfs[cur_h]), slot + a.m_off[cur_h]);
  if (cur_v >= 0) flush(Mv, m_side(a.tfs[cur_v]), slot + a.m_off[cur_v]);
}

// sum over CTAs of the partial sums, in CTA order, in FP64
__global__ void reduce_kernel(const float* partial, int n_ctas, int P, double* M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  double s = 0.0;
  for (int c = 0; c < n_ctas; ++c) s += (double)partial[(size_t)c * P + i];
  M[i] = s;
}

// One CTA per transform with parameters: turns its summed M into the parameter gradient.
//   band:  walk the Givens layers (see below) for dL/dtheta;
//   post:  dL/dQ = M[:K, :K];  dense: dL/dD = M.
__global__ void finish_kernel(const TfDev* tfs, const int* m_off, const int* g_off, const int* kq, const float* P,
                              double* M, float* gparams) {
  const TfDev tf = tfs[blockIdx.x];
  if (tf.kind == KIND_NONE) return;
  double* m = M + m_off[blockIdx.x];
  float* out = gparams + g_off[blockIdx.x];
  if (tf.kind >= KIND_POST) {
    const int K = kq[blockIdx.x], n = tf.kt;
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) out[i] = (float)m[(i / K) * n + (i % K)];
    return;
  }
  // Band A = G_{L-1} ... G_0 with dL/dA = M.  With M_l = (G_{>l})^T M (G_{<l})^T,
  // dL/dtheta for the pair (i, i+1) of layer l is
  //   -s M_l[i][i] - c M_l[i][i+1] + c M_l[i+1][i] - s M_l[i+1][i+1],
  // M_{L-1} = M G_0^T G_1^T ... G_{L-2}^T and M_{l-1} = G_l^T M_l G_{l-1}.
  const int N = tf.n, L = tf.n_layers;
  const float2* cs = reinterpret_cast<const float2*>(P) + tf.cs_off;
  auto layer_off = [&](int l) {
    int off = 0;
    for (int j = 0; j < l; ++j) off += ((j < 32 ? (tf.par_lo >> j) : (tf.par_hi >> (j - 32))) & 1) ? N / 2 - 1 : N / 2;
    return off;
  };
  auto parity = [&](int l) { return (int)(((l < 32 ? (tf.par_lo >> l) : (tf.par_hi >> (l - 32))) & 1)); };
  // right-multiply by G_l^T (mode 0) or G_l (mode 1): mixes columns (i, i+1)
  auto right = [&](int l, int mode) {
    const int par = parity(l), np = (N - par) / 2, off = layer_off(l);
    for (int e = threadIdx.x; e < np * N; e += blockDim.x) {
      const int p = e / N, r = e - p * N, i = 2 * p + par;
      const float2 t = cs[off + p];
      const double c = t.x, s = mode ? -(double)t.y : (double)t.y;
      const double x = m[r * N + i], y = m[r * N + i + 1];
      m[r * N + i] = c * x - s * y;
      m[r * N + i + 1] = s * x + c * y;
    }
    __syncthreads();
  };
  // left-multiply by G_l^T: mixes rows (i, i+1)
  auto left_t = [&](int l) {
    const int par = parity(l), np = (N - par) / 2, off = layer_off(l);
    for (int e = threadIdx.x; e < np * N; e += blockDim.x) {
      const int p = e / N, col = e - p * N, i = 2 * p + par;
      const float2 t = cs[off + p];
      const double c = t.x, s = t.y;
      const double x = m[i * N + col], y = m[(i + 1) * N + col];
      m[i * N + col] = c * x + s * y;
      m[(i + 1) * N + col] = -s * x + c * y;
    }
    __syncthreads();
  };
  for (int l = 0; l + 1 < L; ++l) right(l, 0);
  for (int l = L - 1; l >= 0; --l) {
    const int par = parity(l), np = (N - par) / 2, off = layer_off(l);
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      const int i = 2 * p + par;
      const float2 t = cs[off + p];
      const double c = t.x, s = t.y;
      out[off + p] = (float)(-s * m[i * N + i] - c * m[i * N + i + 1] + c * m[(i + 1) * N + i] -
                             s * m[(i + 1) * N + i + 1]);
    }
    __syncthreads();
    if (l > 0) {
      left_t(l);
      right(l - 1, 1);
    }
  }
}

}  // namespace

int bwd_smem_bytes() { return kBwdSmem; }

const void* bwd_kernel_ptr(bool i16) {
  return i16 ? reinterpret_cast<const void*>(&bwd_kernel<true>) : reinterpret_cast<const void*>(&bwd_kernel<false>);
}

cudaError_t launch_bwd(bool i16, int grid, const BwdArgs& args, double* M, const TfDev* tfs, int n_tfs,
                       const int* m_off, const int* g_off, const int* kq, float* gparams, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(args.partial, 0, (size_t)grid * args.P * sizeof(float), stream);
  if (e != cudaSuccess) return e;
  BwdArgs a = args;
  void* params[] = {&a};
  e = cudaLaunchKernel(bwd_kernel_ptr(i16), dim3(grid), dim3(kBT), params, kBwdSmem, stream);
  if (e != cudaSuccess || !gparams || args.P == 0) return e;
  reduce_kernel<<<(args.P + 255) / 256, 256, 0, stream>>>(args.partial, grid, args.P, M);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finish_kernel<<<n_tfs, 128, 0, stream>>>(tfs, m_off, g_off, kq, args.params, M, gparams);
  return cudaGetLastError();
}

}  // namespace adjtx
