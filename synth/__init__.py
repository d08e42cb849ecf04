"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and bench.py.

This module only draws inputs: AR(1) residual blocks, block lists and random
adjustment parameters.  It holds none of the transform arithmetic, so it can
serve both the CUDA path and the oracle without coupling them.

Residual model: a separable, stationary 2-D AR(1) Gaussian field, the standard
model of prediction residuals that DST-7/DCT-8 style transforms target
(Section 1 of Said, Egilmez & Chao).  For one h x w block, w_{ij} are iid N(0,1);
along each row u_{i,0} = w_{i,0}, u_{i,j} = rho_r u_{i,j-1} + sqrt(1-rho_r^2) w_{i,j};
then along each column v_{0,j} = u_{0,j}, v_{i,j} = rho_c v_{i-1,j} +
sqrt(1-rho_c^2) u_{i,j}; the residual is clip(rint(sigma v), -clip, clip) as int16.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CORE_DCT2, CORE_DCT3, CORE_DST2, CORE_DST3 = 0, 1, 2, 3
KIND_NONE, KIND_BAND, KIND_POST, KIND_DENSE = 0, 1, 2, 3
SIZES = (4, 8, 16, 32, 64)

BLOCK_DTYPE = np.dtype([("offset", "<i8"), ("w", "<u2"), ("h", "<u2"),
                        ("tf_h", "<u2"), ("tf_v", "<u2")])
assert BLOCK_DTYPE.itemsize == 16


@dataclass
class Tf:
    """One 1-D adjusted transform H = C B A of length n."""
    n: int
    core: int
    kind: int = KIND_NONE
    parities: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint8))
    angles: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float64))
    q: np.ndarray | None = None

    @property
    def k(self) -> int:
        return 0 if self.q is None else int(self.q.shape[0])


@dataclass
class Workload:
    name: str
    blocks: np.ndarray          # BLOCK_DTYPE records
    data: np.ndarray            # int16, packed block-linear
    tfs: list
    clip: int
    description: str = ""

    @property
    def total(self) -> int:
        return int(self.data.shape[0])


def n_pairs(n: int, parity: int) -> int:
    return len(range(int(parity), n - 1, 2))


def random_band(rng, n, core, parities, lo=-math.pi / 8, hi=math.pi / 8) -> Tf:
    parities = np.asarray(parities, dtype=np.uint8)
    cnt = sum(n_pairs(n, p) for p in parities)
    return Tf(n=n, core=core, kind=KIND_BAND, parities=parities,
              angles=rng.uniform(lo, hi, size=cnt))


def haar_orthogonal(rng, k: int) -> np.ndarray:
    """Haar-distributed k x k orthogonal matrix: QR of a Gaussian, sign-fixed."""
    Z = rng.standard_normal((k, k))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def random_post(rng, n, core, k) -> Tf:
    return Tf(n=n, core=core, kind=KIND_POST, q=haar_orthogonal(rng, k))


def ar1_blocks(rng, count, h, w, rho_row, rho_col, sigma, clip, chunk=1 << 16):
    """``count`` int16 AR(1) blocks of shape (h, w); rho/sigma scalar or per block."""
    rho_row = np.broadcast_to(np.asarray(rho_row, np.float64), (count,))
    rho_col = np.broadcast_to(np.asarray(rho_col, np.float64), (count,))
    sigma = np.broadcast_to(np.asarray(sigma, np.float64), (count,))
    out = np.empty((count, h, w), dtype=np.int16)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        rr = rho_row[s:e, None]
        rc = rho_col[s:e, None]
        u = rng.standard_normal((e - s, h, w))
        gr = np.sqrt(1.0 - rr * rr)
        for j in range(1, w):
            u[:, :, j] = rr * u[:, :, j - 1] + gr * u[:, :, j]
        gc = np.sqrt(1.0 - rc * rc)
        for i in range(1, h):
            u[:, i, :] = rc * u[:, i - 1, :] + gc * u[:, i, :]
        x = np.rint(sigma[s:e, None, None] * u)
        np.clip(x, -clip, clip, out=x)
        out[s:e] = x.astype(np.int16)
    return out


def _pack(sizes_tfs, rng, stats, clip):
    """Build the block list and residual buffer for blocks given in order.

    sizes_tfs: int arrays (w, h, tf_h, tf_v), one entry per block, in storage
    order.  stats(rng, count) -> (rho_row, rho_col, sigma) arrays for count blocks.
    """
    w, h, th, tv = (np.asarray(a) for a in sizes_tfs)
    nb = w.shape[0]
    blocks = np.zeros(nb, dtype=BLOCK_DTYPE)
    sz = (w.astype(np.int64) * h.astype(np.int64))
    off = np.zeros(nb, dtype=np.int64)
    if nb:
        off[1:] = np.cumsum(sz)[:-1]
    blocks["offset"], blocks["w"], blocks["h"] = off, w, h
    blocks["tf_h"], blocks["tf_v"] = th, tv
    total = int(sz.sum())
    data = np.empty(total, dtype=np.int16)
    # Per-block statistics are drawn in storage order, then the fields are
    # generated per size class (vectorised) from a child stream.
    rr, rc, sg = stats(rng, nb)
    gen = np.random.Generator(np.random.PCG64(rng.integers(1 << 62)))
    for ww, hh in sorted(set(zip(w.tolist(), h.tolist()))):
        sel = np.nonzero((w == ww) & (h == hh))[0]
        blk = ar1_blocks(gen, sel.size, hh, ww, rr[sel], rc[sel], sg[sel], clip)
        idx = off[sel, None] + np.arange(ww * hh)[None, :]
        data[idx] = blk.reshape(sel.size, -1)
    return blocks, data


def _stats_c2(rng, nb):
    return (rng.uniform(0.6, 0.99, nb), rng.uniform(0.6, 0.99, nb),
            np.exp(3.0 + rng.standard_normal(nb)))


def blocks32_band(seed: int = 1) -> Workload:
    """1024 blocks 32x32, rho=0.95, sigma=40, clip 255; DCT-2 + 2-layer band both ways."""
    rng = np.random.default_rng(seed)
    tfs = [random_band(rng, 32, CORE_DCT2, [0, 1]),   # horizontal
           random_band(rng, 32, CORE_DCT2, [0, 1])]   # vertical
    nb = 1024
    data = ar1_blocks(rng, nb, 32, 32, 0.95, 0.95, 40.0, 255).reshape(-1)
    blocks = np.zeros(nb, dtype=BLOCK_DTYPE)
    blocks["offset"] = np.arange(nb, dtype=np.int64) * 1024
    blocks["w"] = blocks["h"] = 32
    blocks["tf_h"], blocks["tf_v"] = 0, 1
    return Workload("1024x32x32-dct2-band2", blocks, data, tfs, 255,
                    "1024 32x32 AR(1) rho=.95 sigma=40; DCT-2 + 2-layer band, both directions")


def blocks32_64_mixed(seed: int = 2, per_size: int = 2048) -> Workload:
    """2048 x 32x32 + 2048 x 64x64, 10-bit; H: DST-3 + 4-layer band; V: DCT-2 + post K=N/2."""
    rng = np.random.default_rng(seed)
    tfs = []
    ids = {}
    for n in (32, 64):
        ids[("h", n)] = len(tfs)
        tfs.append(random_band(rng, n, CORE_DST3, [0, 1, 0, 1]))
        ids[("v", n)] = len(tfs)
        tfs.append(random_post(rng, n, CORE_DCT2, n // 2))
    w = np.array([32] * per_size + [64] * per_size)
    th = np.array([ids[("h", int(x))] for x in w])
    tv = np.array([ids[("v", int(x))] for x in w])
    blocks, data = _pack((w, w, th, tv), rng, _stats_c2, 1023)
    return Workload(f"{per_size}x32x32+{per_size}x64x64-dst3band4-dct2post", blocks,
                    data, tfs, 1023,
                    "2048x32x32 + 2048x64x64 10-bit AR(1), rho~U[.6,.99], sigma~logN(3,1); "
                    "H DST-3 + 4-layer band, V DCT-2 + post K=N/2")


def mixed_tf_table(rng):
    """One parameter set per (direction, N, core, kind): band = 4 layers, post K = N/2."""
    tfs, ids = [], {}
    for d in ("h", "v"):
        for n in SIZES:
            for core in range(4):
                for kind in range(3):
                    ids[(d, n, core, kind)] = len(tfs)
                    if kind == KIND_NONE:
                        tfs.append(Tf(n=n, core=core))
                    elif kind == KIND_BAND:
                        tfs.append(random_band(rng, n, core, [0, 1, 0, 1]))
                    else:
                        tfs.append(random_post(rng, n, core, n // 2))
    return tfs, ids


_CTU_P = np.array([1 / 6, 1 / 6, 1 / 6, 0.35, 0.15])


def _ctu_sizes(rng, frames: int, width: int, height: int):
    """Block widths and heights of frames tiled into 64x64 CTUs, per-CTU sizes.

    W and H are drawn per CTU from {4,...,64} (P(64)=.15, P(32)=.35, rest 1/6);
    the CTU is tiled uniformly by W x H blocks in raster order.  A partial CTU
    row at the bottom (2160 = 33*64 + 48) is split into power-of-two regions
    (32 then 16) with H clamped to the region height.
    """
    cols = width // 64
    full_rows, rem = divmod(height, 64)
    regions = []                      # heights of the bottom strip regions
    r = rem
    for s in (32, 16, 8, 4):
        if r >= s:
            regions.append(s)
            r -= s
    assert r == 0, "frame height must be a multiple of 4"
    ws, hs = [], []
    sizes = np.array(SIZES)
    for _f in range(frames):
        for cy in range(full_rows + (1 if rem else 0)):
            reg = [64] if cy < full_rows else regions
            for _cx in range(cols):
                W = int(rng.choice(sizes, p=_CTU_P))
                H = int(rng.choice(sizes, p=_CTU_P))
                for rh in reg:
                    hh = min(H, rh)
                    n = (64 // W) * (rh // hh)
                    ws.extend([W] * n)
                    hs.extend([hh] * n)
    return np.array(ws), np.array(hs)


def uhd_mixed(seed: int = 3, frames: int = 8, width: int = 3840, height: int = 2160) -> Workload:
    """Frames tiled into CTUs of 64x64 with per-CTU block sizes (``_ctu_sizes``),
    per-block types: each block draws its horizontal and vertical (core, kind)
    uniformly from the 12 combinations.
    """
    rng = np.random.default_rng(seed)
    tfs, ids = mixed_tf_table(rng)
    w, h = _ctu_sizes(rng, frames, width, height)
    nb = w.size
    ch = rng.integers(0, 4, nb)
    kh = rng.integers(0, 3, nb)
    cv = rng.integers(0, 4, nb)
    kv = rng.integers(0, 3, nb)
    lut_h = np.full((65, 4, 3), -1)
    lut_v = np.full((65, 4, 3), -1)
    for (d, n, c, k), i in ids.items():
        (lut_h if d == "h" else lut_v)[n, c, k] = i
    th = lut_h[w, ch, kh]
    tv = lut_v[h, cv, kv]
    blocks, data = _pack((w, h, th, tv), rng, _stats_c2, 1023)
    return Workload(f"mixed4-64-{frames}x{width}x{height}", blocks, data, tfs, 1023,
                    f"{frames} frames {width}x{height} tiled by per-CTU sizes 4..64, "
                    "per-block core x adjustment in each direction, 10-bit AR(1)")


FRAME_BLOCK_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("w", "<u2"), ("h", "<u2"),
                              ("tf_h", "<u2"), ("tf_v", "<u2")])


def ctu_frame_blocks(rng, width: int, height: int):
    """Positions and sizes of the blocks of one frame tiled like the mixed UHD workload (``_ctu_sizes``):
    (x, y, w, h) arrays, CTUs in raster order, blocks in raster order inside a CTU region."""
    cols = width // 64
    full_rows, rem = divmod(height, 64)
    regions = []
    r = rem
    for s in (32, 16, 8, 4):
        if r >= s:
            regions.append(s)
            r -= s
    assert r == 0, "frame height must be a multiple of 4"
    sizes = np.array(SIZES)
    xs, ys, ws, hs = [], [], [], []
    for cy in range(full_rows + (1 if rem else 0)):
        reg = [64] if cy < full_rows else regions
        for cx in range(cols):
            W = int(rng.choice(sizes, p=_CTU_P))
            H = int(rng.choice(sizes, p=_CTU_P))
            y0 = cy * 64
            for rh in reg:
                hh = min(H, rh)
                for by in range(rh // hh):
                    for bx in range(64 // W):
                        xs.append(cx * 64 + bx * W)
                        ys.append(y0 + by * hh)
                        ws.append(W)
                        hs.append(hh)
                y0 += rh
    return np.array(xs), np.array(ys), np.array(ws), np.array(hs)


def uhd_mixed_frame(seed: int = 3, width: int = 3840, height: int = 2160, stride: int | None = None,
                    frames: int = 1):
    """Mixed UHD frames in frame layout: (frame int16 [frames * height, stride], frame blocks, tfs).

    The blocks tile each frame as in ``uhd_mixed`` (per-CTU sizes, per-block core x adjustment in
    each direction, 10-bit AR(1) residual per block); ``stride`` (default: width rounded up to
    a multiple of 64) leaves unused samples at the end of every row.  Several frames are
    stacked one below the other, which makes them one taller frame with the same stride."""
    rng = np.random.default_rng(seed)
    tfs, ids = mixed_tf_table(rng)
    parts = [ctu_frame_blocks(rng, width, height) for _ in range(frames)]
    x = np.concatenate([p[0] for p in parts])
    y = np.concatenate([p[1] + f * height for f, p in enumerate(parts)])
    w = np.concatenate([p[2] for p in parts])
    h = np.concatenate([p[3] for p in parts])
    nb = w.size
    ch, kh = rng.integers(0, 4, nb), rng.integers(0, 3, nb)
    cv, kv = rng.integers(0, 4, nb), rng.integers(0, 3, nb)
    lut_h = np.full((65, 4, 3), -1)
    lut_v = np.full((65, 4, 3), -1)
    for (d, n, c, k), i in ids.items():
        (lut_h if d == "h" else lut_v)[n, c, k] = i
    packed, data = _pack((w, h, lut_h[w, ch, kh], lut_v[h, cv, kv]), rng, _stats_c2, 1023)
    stride = stride or (width + 63) // 64 * 64
    frame = np.zeros((frames * height, stride), dtype=np.int16)
    blocks = np.zeros(nb, dtype=FRAME_BLOCK_DTYPE)
    blocks["x"], blocks["y"], blocks["w"], blocks["h"] = x, y, w, h
    blocks["tf_h"], blocks["tf_v"] = packed["tf_h"], packed["tf_v"]
    for (ww, hh) in sorted(set(zip(w.tolist(), h.tolist()))):
        sel = np.nonzero((w == ww) & (h == hh))[0]
        vals = data[packed["offset"][sel, None] + np.arange(ww * hh)[None, :]].reshape(-1, hh, ww)
        rows = y[sel, None, None] + np.arange(hh)[None, :, None]
        cols = x[sel, None, None] + np.arange(ww)[None, None, :]
        frame[rows, cols] = vals
    return frame, blocks, tfs


def uhd_mixed_multiple(seed: int = 3, frames: int = 8, width: int = 3840, height: int = 2160,
                       k_max: int = 8) -> Workload:
    """The mixed UHD frame tiling for the encoder's DST-7 / DCT-8 search (Section 2.3):
    every block uses, in each direction, a DCT-2 with a post-adjustment of size
    K = min(k_max, n/2) (the 8 x 8 adjustment at 16 points and more), Q Haar-random per
    (direction, n).  Same residual statistics as ``uhd_mixed``."""
    rng = np.random.default_rng(seed)
    tfs, lut = [], {}
    for d in ("h", "v"):
        for n in SIZES:
            lut[d, n] = len(tfs)
            tfs.append(random_post(rng, n, CORE_DCT2, min(k_max, n // 2)))
    w, h = _ctu_sizes(rng, frames, width, height)
    th = np.array([lut["h", int(x)] for x in SIZES])[np.log2(w).astype(int) - 2]
    tv = np.array([lut["v", int(x)] for x in SIZES])[np.log2(h).astype(int) - 2]
    blocks, data = _pack((w, h, th, tv), rng, _stats_c2, 1023)
    return Workload(f"mixed4-64-multiple-{frames}x{width}x{height}", blocks, data, tfs, 1023,
                    f"{frames} frames {width}x{height} tiled by per-CTU sizes 4..64, DCT-2 + "
                    f"K=min({k_max}, n/2) post-adjustment both ways, 10-bit AR(1)")


def uhd8k(seed: int = 5, frames: int = 16, width: int = 7680, height: int = 4320,
          h_tf: Tf | None = None, v_tfs: dict | None = None) -> Workload:
    """All 64x64 / 64x32 blocks; H: DST-3 + band at 64, V: DCT-2 + post (K=32 @64, 16 @32).

    Each full CTU is one 64x64 block or, with probability 1/2, two 64x32; the
    final 32-row strip is 64x32.  ``h_tf``/``v_tfs`` override the seeded
    parameters (e.g. with fitted ones).
    """
    rng = np.random.default_rng(seed)
    if h_tf is None:
        h_tf = random_band(rng, 64, CORE_DST3, [0, 1] * 6)
    if v_tfs is None:
        v_tfs = {64: random_post(rng, 64, CORE_DCT2, 32), 32: random_post(rng, 32, CORE_DCT2, 16)}
    tfs = [h_tf, v_tfs[64], v_tfs[32]]
    cols = width // 64
    full_rows, rem = divmod(height, 64)
    assert rem in (0, 32)
    split = rng.random((frames, full_rows, cols)) < 0.5
    hs = []
    for f in range(frames):
        for cy in range(full_rows):
            for cx in range(cols):
                hs.extend([32, 32] if split[f, cy, cx] else [64])
        if rem:
            hs.extend([32] * cols)
    h = np.array(hs)
    w = np.full_like(h, 64)
    th = np.zeros_like(h)
    tv = np.where(h == 64, 1, 2)
    blocks, data = _pack((w, h, th, tv), rng, _stats_c2, 1023)
    return Workload(f"64x64+64x32-{frames}x{width}x{height}", blocks, data, tfs, 1023,
                    f"{frames} frames {width}x{height}, 64x64 and 64x32 blocks; H DST-3 + "
                    "12-layer band, V DCT-2 + post K=N/2, 10-bit AR(1)")


def random_small(seed: int, n_blocks: int, clip: int = 1023) -> Workload:
    """Fuzz workload: random sizes, random types per direction, odd batch sizes."""
    rng = np.random.default_rng(seed)
    tfs, ids = mixed_tf_table(rng)
    sizes = np.array(SIZES)
    w = rng.choice(sizes, n_blocks)
    h = rng.choice(sizes, n_blocks)
    lut_h = np.full((65, 4, 3), -1)
    lut_v = np.full((65, 4, 3), -1)
    for (d, n, c, k), i in ids.items():
        (lut_h if d == "h" else lut_v)[n, c, k] = i
    th = lut_h[w, rng.integers(0, 4, n_blocks), rng.integers(0, 3, n_blocks)]
    tv = lut_v[h, rng.integers(0, 4, n_blocks), rng.integers(0, 3, n_blocks)]
    blocks, data = _pack((w, h, th, tv), rng, _stats_c2, clip)
    return Workload(f"random-{seed}-{n_blocks}", blocks, data, tfs, clip, "fuzz")

