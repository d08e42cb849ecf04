"""Plain FP64 oracle of the adjusted 2-D transforms.

TEST INFRASTRUCTURE.  This module is the reference the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs
of ``bench.py`` may use it; it shares no code with the CUDA library and imports
nothing from it.

Source: A. Said, H. E. Egilmez, Y.-H. Chao, "Low-complexity transform
adjustments for video coding".

Conventions (all in float64):

* A transform matrix has the frequency index k along its rows and the sample
  index n along its columns; the forward 1-D transform of a line x is y = T x
  and its inverse is x = T^T y (every matrix here is orthogonal).
* Cores B are the orthonormal DCT-2, DCT-3, DST-2 and DST-3 (Section 2.1),
  written from their closed forms.  The DST-7 / DCT-8 targets D of Section 2.2
  (Eq. 3) are written from theirs.
* The adjusted 1-D transform is H = C B A (Eq. 1).  A is a band matrix made of
  layers of disjoint adjacent-pair Givens rotations (Section 2, after Eq. 2, and
  Section 2.2); layer 0 touches the input first, an even layer rotates pairs
  (0,1),(2,3),..., an odd layer rotates (1,2),(3,4),...,(N-3,N-2), and a
  rotation by theta maps (x_i, x_{i+1}) to (c x_i - s x_{i+1}, s x_i + c x_{i+1}).
  C = diag(Q, I_{N-K}) is the top-left K x K post-adjustment (Section 2.2,
  Section 2.3: only the first K outputs change).
* A block is stored row-major with h rows and w columns.  The horizontal
  transform H_h (w x w) acts along each row, the vertical H_v (h x h) along each
  column: Y = H_v X H_h^T, and the inverse is X = H_v^T Y H_h (Section 2.2: the
  adjustments act horizontally and vertically on the whole block).

Every function is the definition written out; numpy matmul is the only library
step.  There is no blocking, fusion or reordering of the arithmetic beyond
grouping independent blocks that use the same matrices into one batched
matmul.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "CORE_DCT2", "CORE_DCT3", "CORE_DST2", "CORE_DST3",
    "KIND_NONE", "KIND_BAND", "KIND_POST", "KIND_DENSE",
    "dct2", "dct3", "dst2", "dst3", "dst7", "dct8", "dct4",
    "reversal", "alt_sign", "core_matrix",
    "layer_pairs", "givens_layer", "band_matrix", "post_matrix",
    "adjusted_matrix", "tf_matrix",
    "forward_2d", "inverse_2d", "forward_blocks", "inverse_blocks",
    "dct2_fast", "dct4_fast",
    "eq2_weighted_error",
]

CORE_DCT2, CORE_DCT3, CORE_DST2, CORE_DST3 = 0, 1, 2, 3
KIND_NONE, KIND_BAND, KIND_POST, KIND_DENSE = 0, 1, 2, 3


# --------------------------------------------------------------------------
# Closed-form trigonometric matrices (Section 1, Section 2.1, Section 2.2).
# Orthonormal scaling throughout: c_0 = 1/sqrt(2) for the cosine families,
# d_{N-1} = 1/sqrt(2) for the sine families.
# --------------------------------------------------------------------------

def _kn(N):
    k = np.arange(N, dtype=np.float64)[:, None]
    n = np.arange(N, dtype=np.float64)[None, :]
    return k, n


def dct2(N: int) -> np.ndarray:
    """DCT-2: T[k,n] = c_k sqrt(2/N) cos(pi (2n+1) k / (2N))."""
    k, n = _kn(N)
    T = math.sqrt(2.0 / N) * np.cos(np.pi * (2 * n + 1) * k / (2 * N))
    T[0, :] *= 1.0 / math.sqrt(2.0)
    return T


def dct3(N: int) -> np.ndarray:
    """DCT-3: T[k,n] = c_n sqrt(2/N) cos(pi (2k+1) n / (2N))."""
    k, n = _kn(N)
    T = math.sqrt(2.0 / N) * np.cos(np.pi * (2 * k + 1) * n / (2 * N))
    T[:, 0] *= 1.0 / math.sqrt(2.0)
    return T


def dst2(N: int) -> np.ndarray:
    """DST-2: T[k,n] = d_k sqrt(2/N) sin(pi (2n+1) (k+1) / (2N))."""
    k, n = _kn(N)
    T = math.sqrt(2.0 / N) * np.sin(np.pi * (2 * n + 1) * (k + 1) / (2 * N))
    T[N - 1, :] *= 1.0 / math.sqrt(2.0)
    return T


def dst3(N: int) -> np.ndarray:
    """DST-3: T[k,n] = d_n sqrt(2/N) sin(pi (2k+1) (n+1) / (2N))."""
    k, n = _kn(N)
    T = math.sqrt(2.0 / N) * np.sin(np.pi * (2 * k + 1) * (n + 1) / (2 * N))
    T[:, N - 1] *= 1.0 / math.sqrt(2.0)
    return T


def dst7(N: int) -> np.ndarray:
    """DST-7 (Section 2.2): T[k,n] = sqrt(4/(2N+1)) sin(pi (2k+1)(n+1) / (2N+1)).

    The basis index k multiplies (2k+1); the transposed reading is the DST-6
    and fails Eq. 3 against the DCT-8 below.
    """
    k, n = _kn(N)
    return math.sqrt(4.0 / (2 * N + 1)) * np.sin(np.pi * (2 * k + 1) * (n + 1) / (2 * N + 1))


def dct8(N: int) -> np.ndarray:
    """DCT-8 (Section 2.2): T[k,n] = sqrt(4/(2N+1)) cos(pi (2k+1)(2n+1) / (4N+2))."""
    k, n = _kn(N)
    return math.sqrt(4.0 / (2 * N + 1)) * np.cos(np.pi * (2 * k + 1) * (2 * n + 1) / (4 * N + 2))


def dct4(N: int) -> np.ndarray:
    """DCT-4: T[k,n] = sqrt(2/N) cos(pi (2n+1)(2k+1) / (4N)) (odd half of the DCT-2)."""
    k, n = _kn(N)
    return math.sqrt(2.0 / N) * np.cos(np.pi * (2 * n + 1) * (2 * k + 1) / (4 * N))


def reversal(N: int) -> np.ndarray:
    """R of Section 2.1: R[m,n] = 1 iff m = N-1-n."""
    R = np.zeros((N, N))
    R[np.arange(N), N - 1 - np.arange(N)] = 1.0
    return R


def alt_sign(N: int) -> np.ndarray:
    """S of Section 2.1: diagonal with S[m,m] = (-1)^m."""
    return np.diag((-1.0) ** np.arange(N))


_CORES = {CORE_DCT2: dct2, CORE_DCT3: dct3, CORE_DST2: dst2, CORE_DST3: dst3}


def core_matrix(N: int, core: int) -> np.ndarray:
    """The fast core B (Section 2.1) as its closed-form matrix."""
    return _CORES[int(core)](N)


# --------------------------------------------------------------------------
# Adjustments (Eq. 1; Givens factorisation after Eq. 2; Section 2.2).
# --------------------------------------------------------------------------

def layer_pairs(N: int, parity: int):
    """Index pairs (i, i+1) rotated by one layer: even from 0, odd from 1, no wrap."""
    return [(i, i + 1) for i in range(int(parity), N - 1, 2)]


def givens_layer(N: int, parity: int, angles) -> np.ndarray:
    """One layer of parallel adjacent-pair Givens rotations as an N x N matrix."""
    pairs = layer_pairs(N, parity)
    angles = np.asarray(angles, dtype=np.float64)
    if angles.shape != (len(pairs),):
        raise ValueError(f"layer of parity {parity} at N={N} needs {len(pairs)} angles")
    G = np.eye(N)
    for (i, j), th in zip(pairs, angles):
        c, s = math.cos(th), math.sin(th)
        G[i, i], G[i, j] = c, -s
        G[j, i], G[j, j] = s, c
    return G


def band_matrix(N: int, parities, angles) -> np.ndarray:
    """A = G_{L-1} ... G_1 G_0; the angles of layer 0 come first in ``angles``."""
    angles = np.asarray(angles, dtype=np.float64).ravel()
    A = np.eye(N)
    pos = 0
    for p in parities:
        cnt = len(layer_pairs(N, int(p)))
        A = givens_layer(N, int(p), angles[pos:pos + cnt]) @ A
        pos += cnt
    if pos != angles.size:
        raise ValueError(f"{angles.size} angles given, layers need {pos}")
    return A


def post_matrix(N: int, Q) -> np.ndarray:
    """C = diag(Q, I_{N-K}): Q acts on the K lowest-frequency outputs."""
    Q = np.asarray(Q, dtype=np.float64)
    K = Q.shape[0]
    if Q.shape != (K, K) or K > N:
        raise ValueError("Q must be K x K with K <= N")
    C = np.eye(N)
    C[:K, :K] = Q
    return C


def adjusted_matrix(N, core, kind, parities=(), angles=(), Q=None) -> np.ndarray:
    """H = C B A of Eq. 1 for one direction."""
    B = core_matrix(N, core)
    if kind == KIND_NONE:
        return B
    if kind == KIND_BAND:
        return B @ band_matrix(N, parities, angles)
    if kind == KIND_POST:
        return post_matrix(N, Q) @ B
    if kind == KIND_DENSE:
        # the reference the adjustments approximate: a given dense orthogonal matrix D
        Q = np.asarray(Q, dtype=np.float64)
        if Q.shape != (N, N):
            raise ValueError("a dense transform is N x N")
        return Q.copy()
    raise ValueError(f"unknown adjustment kind {kind}")


def tf_matrix(tf) -> np.ndarray:
    """H for an object (or dict) carrying n, core, kind, parities, angles, q."""
    get = (lambda k: tf[k]) if isinstance(tf, dict) else (lambda k: getattr(tf, k))
    kind = int(get("kind"))
    return adjusted_matrix(
        int(get("n")), int(get("core")), kind,
        parities=get("parities") if kind == KIND_BAND else (),
        angles=get("angles") if kind == KIND_BAND else (),
        Q=get("q") if kind in (KIND_POST, KIND_DENSE) else None,
    )


# --------------------------------------------------------------------------
# Separable 2-D application (Section 2.2).
# --------------------------------------------------------------------------

def forward_2d(X, Hh, Hv) -> np.ndarray:
    """Y = H_v X H_h^T for one block or a stack of blocks (..., h, w)."""
    X = np.asarray(X, dtype=np.float64)
    return Hv @ X @ Hh.T


def inverse_2d(Y, Hh, Hv) -> np.ndarray:
    """X = H_v^T Y H_h, the inverse of ``forward_2d`` for orthogonal H."""
    Y = np.asarray(Y, dtype=np.float64)
    return Hv.T @ Y @ Hh


def _apply_blocks(src, blocks, tfs, fn):
    src = np.asarray(src)
    out = np.zeros(src.shape[0], dtype=np.float64)
    mats = {}

    def H(i):
        if i not in mats:
            mats[i] = tf_matrix(tfs[i])
        return mats[i]

    off = np.asarray(blocks["offset"], dtype=np.int64)
    key = np.stack([np.asarray(blocks[f], dtype=np.int64)
                    for f in ("w", "h", "tf_h", "tf_v")], axis=1)
    if key.shape[0] == 0:
        return out
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    for g, (w, h, th, tv) in enumerate(uniq):
        sel = off[inv == g]
        idx = sel[:, None] + np.arange(w * h)[None, :]
        X = src[idx].astype(np.float64).reshape(-1, h, w)
        out[idx] = fn(X, H(int(th)), H(int(tv))).reshape(-1, w * h)
    return out


def forward_blocks(x_flat, blocks, tfs) -> np.ndarray:
    """FP64 forward transform of every block of a packed block-linear buffer.

    ``blocks`` has fields offset, w, h, tf_h, tf_v; ``tfs[i]`` describes 1-D
    transform i.  Positions not covered by a block are left at zero.
    """
    return _apply_blocks(x_flat, blocks, tfs, forward_2d)


def inverse_blocks(y_flat, blocks, tfs) -> np.ndarray:
    """FP64 inverse transform of every block (see ``forward_blocks``)."""
    return _apply_blocks(y_flat, blocks, tfs, inverse_2d)


# --------------------------------------------------------------------------
# The oracle's own FP64 fast DCT-2 (Section 1 / 2.1: the even/odd structure that
# makes the DCT-2 family cheap).  Checked against the closed form in the tests.
# --------------------------------------------------------------------------

def dct2_fast(x) -> np.ndarray:
    """Orthonormal DCT-2 of a line by even/odd recursion.

    The even outputs are the half-length DCT-2 of (x_n + x_{N-1-n})/sqrt(2);
    the odd outputs are the half-length DCT-4 of (x_n - x_{N-1-n})/sqrt(2).
    """
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[-1]
    if N == 1:
        return x.copy()
    h = N // 2
    head, tail = x[..., :h], x[..., ::-1][..., :h]
    y = np.empty_like(x)
    y[..., 0::2] = dct2_fast((head + tail) / math.sqrt(2.0))
    y[..., 1::2] = dct4_fast((head - tail) / math.sqrt(2.0))
    return y


def dct4_fast(x) -> np.ndarray:
    """Orthonormal DCT-4 of length M via an M/2-point complex DFT.

    Pair a_m = x_{2m} with b_m = x_{M-1-2m}, form z_m = (a_m - i b_m) e^{i pi m / M},
    take Z_p = sum_m z_m e^{2 pi i m p / (M/2)} and W_p = sqrt(2/M) Z_p
    e^{i pi (4p+1) / (4M)}; then X_{2p} = Re W_p and X_{M-1-2p} = Im W_p.
    """
    x = np.asarray(x, dtype=np.float64)
    M = x.shape[-1]
    if M == 1:
        return x.copy()
    P = M // 2
    m = np.arange(P)
    a = x[..., 2 * m]
    b = x[..., M - 1 - 2 * m]
    z = (a - 1j * b) * np.exp(1j * np.pi * m / M)
    Z = np.fft.ifft(z, axis=-1) * P
    W = math.sqrt(2.0 / M) * Z * np.exp(1j * np.pi * (4 * m + 1) / (4 * M))
    X = np.empty_like(x)
    X[..., 2 * m] = W.real
    X[..., M - 1 - 2 * m] = W.imag
    return X


# --------------------------------------------------------------------------
# Design criterion (Eq. 2).
# --------------------------------------------------------------------------

def eq2_weighted_error(H, D) -> float:
    """sum_i sum_j e^{-alpha i} (H_ij - D_ij)^2 with alpha = ln(10^2)/N (Eq. 2)."""
    H = np.asarray(H, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    N = H.shape[0]
    alpha = math.log(100.0) / N
    w = np.exp(-alpha * np.arange(N))[:, None]
    return float(np.sum(w * (H - D) ** 2))


# --------------------------------------------------------------------------
# Gradients (design of the adjustments, Eq. 2 and the Givens factorisation after
# it; Section 2.2).  Everything is FP64 and follows the chain rule term by term.
# --------------------------------------------------------------------------

def grad_2d(X, G, Hh, Hv):
    """For Y = H_v X H_h^T and upstream G = dL/dY (stacks (..., h, w)):
    returns (dL/dX, dL/dH_h, dL/dH_v) with dL/dX = H_v^T G H_h,
    dL/dH_h = sum_b G_b^T H_v X_b and dL/dH_v = sum_b G_b H_h X_b^T."""
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    gX = Hv.T @ G @ Hh
    Xb = X.reshape((-1,) + X.shape[-2:])
    Gb = G.reshape((-1,) + G.shape[-2:])
    dHh = np.einsum("bji,jk,bkl->il", Gb, Hv, Xb)
    dHv = np.einsum("bij,jk,blk->il", Gb, Hh, Xb)
    return gX, dHh, dHv


def grad_band_angles(N, core, parities, angles, dH):
    """dL/dtheta for H = B G_{L-1} ... G_0 given dL/dH.

    dL/dtheta_j = < dL/dH , B G_{L-1} .. G_{l+1} (dG_l/dtheta_j) G_{l-1} .. G_0 >,
    where layer l holds rotation j and dG_l/dtheta_j is zero except for its 2x2 block
    [[-s, -c], [c, -s]]."""
    angles = np.asarray(angles, dtype=np.float64).ravel()
    B = core_matrix(N, core)
    layers, pos = [], 0
    for p in parities:
        cnt = len(layer_pairs(N, int(p)))
        layers.append((int(p), angles[pos:pos + cnt]))
        pos += cnt
    Gs = [givens_layer(N, p, a) for p, a in layers]
    out = np.zeros_like(angles)
    pos = 0
    for l, (p, a) in enumerate(layers):
        left = B.copy()
        for m in range(len(Gs) - 1, l, -1):
            left = left @ Gs[m]
        right = np.eye(N)
        for m in range(l):
            right = Gs[m] @ right
        M = left.T @ dH @ right.T          # dL/dG_l
        for q, ((i, j), th) in enumerate(zip(layer_pairs(N, p), a)):
            c, s = math.cos(th), math.sin(th)
            out[pos + q] = -s * M[i, i] - c * M[i, j] + c * M[j, i] - s * M[j, j]
        pos += len(a)
    return out


def grad_post_q(N, core, K, dH):
    """dL/dQ for H = diag(Q, I) B: the top-left K x K block of dL/dH B^T."""
    B = core_matrix(N, core)
    return (dH @ B.T)[:K, :K]


def skew_from_params(w, K):
    """K x K skew-symmetric W from its K(K-1)/2 upper-triangle entries (row major)."""
    W = np.zeros((K, K))
    iu = np.triu_indices(K, 1)
    W[iu] = np.asarray(w, dtype=np.float64)
    return W - W.T


def cayley(w, K, D=None):
    """Q = D (I + W)^{-1} (I - W): orthogonal with det = det(D) (D a fixed +-1 diagonal)."""
    W = skew_from_params(w, K)
    I = np.eye(K)
    Q = np.linalg.solve(I + W, I - W)
    if D is not None:
        Q = np.diag(D) @ Q
    return Q


def cayley_grad(w, K, GQ, D=None):
    """dL/dw for Q = D Cayley(W): with C = Cayley(W) and G_C = D^T dL/dQ,
    dL/dW_full = -(I + W)^{-T} G_C (C + I)^T and dL/dw_ij = M_ij - M_ji (i < j)."""
    W = skew_from_params(w, K)
    I = np.eye(K)
    C = np.linalg.solve(I + W, I - W)
    GC = np.asarray(GQ, dtype=np.float64)
    if D is not None:
        GC = np.diag(D) @ GC
    M = -np.linalg.solve((I + W).T, GC) @ (C + I).T
    iu = np.triu_indices(K, 1)
    return (M - M.T)[iu]


def basis_loss(H, D, M):
    """sum_{k<M} |h_k - d_k|^2 over the first M rows (basis vectors) and its dL/dH."""
    H = np.asarray(H, dtype=np.float64)
    diff = np.zeros_like(H)
    diff[:M] = H[:M] - np.asarray(D, dtype=np.float64)[:M]
    return float(np.sum(diff ** 2)), 2.0 * diff


def proxy_loss(Y):
    """Coding-gain proxy (1/(h w)) sum_{kv,kh} log(mean_b Y_b[kv,kh]^2) over a stack of
    coefficient blocks, and its dL/dY."""
    Y = np.asarray(Y, dtype=np.float64)
    nb = Y.shape[0]
    var = np.mean(Y ** 2, axis=0)
    hw = Y.shape[1] * Y.shape[2]
    L = float(np.sum(np.log(var)) / hw)
    G = (2.0 / (hw * nb)) * Y / var[None]
    return L, G


__all__ += ["grad_2d", "grad_band_angles", "grad_post_q", "skew_from_params", "cayley",
            "cayley_grad", "basis_loss", "proxy_loss"]


# --------------------------------------------------------------------------
# Simultaneous DST-7 and DCT-8 adjustments for the encoder search (Section 2.3).
#
# With a top-left post-adjustment after the DCT-2, S T^(C2) = T^(C2) R turns Eq. 3 into
# Eq. 5: the DCT-8 adjustment is C^(C8) = S C^(S7) S.  An encoder that tries the 2-D
# DCT-2 and every (vertical, horizontal) pairing of DST-7 and DCT-8 therefore needs one
# DCT-2 per line plus the K x K products of the first K outputs; every other coefficient
# of the four adjusted transforms equals the DCT-2 one.
# --------------------------------------------------------------------------

# (vertical, horizontal) pairings in output order; "S" = DST-7 adjustment, "C" = DCT-8.
MULTI_COMBOS = ("SS", "SC", "CS", "CC")


def post_c8_from_s7(Q) -> np.ndarray:
    """K x K block of C^(C8) = S C^(S7) S (Eq. 5): Q with entry (i, j) times (-1)^(i+j)."""
    Q = np.asarray(Q, dtype=np.float64)
    S = alt_sign(Q.shape[0])
    return S @ Q @ S


def multiple_1d(N: int, Q=None):
    """(T^(C2), C^(S7) T^(C2), C^(C8) T^(C2)) for C^(S7) = diag(Q, I); Q None means K = 0
    (no adjustment: all three are the DCT-2).  C^(C8) is formed as S C^(S7) S with the N x N
    sign matrix, exactly as Eq. 5 states it."""
    B = dct2(N)
    if Q is None or np.asarray(Q).size == 0:
        return B, B.copy(), B.copy()
    C = post_matrix(N, Q)
    S = alt_sign(N)
    return B, C @ B, S @ C @ S @ B


def multiple_2d(X, Qh=None, Qv=None) -> dict:
    """Y_DD = T_v X T_h^T (2-D DCT-2) and Y_ab = H_a^v X (H_b^h)^T for every pairing ab of
    MULTI_COMBOS (a vertical, b horizontal), each by its own dense product."""
    X = np.asarray(X, dtype=np.float64)
    h, w = X.shape[-2:]
    Dh, Sh, Ch = multiple_1d(w, Qh)
    Dv, Sv, Cv = multiple_1d(h, Qv)
    hor = {"S": Sh, "C": Ch}
    ver = {"S": Sv, "C": Cv}
    out = {"DD": forward_2d(X, Dh, Dv)}
    for ab in MULTI_COMBOS:
        out[ab] = forward_2d(X, hor[ab[1]], ver[ab[0]])
    return out


def multiple_side_size(w: int, h: int, kh: int, kv: int) -> int:
    """Floats of one block's distinct adjusted coefficients (layout of ``multiple_side``):
    2 kv (w - kh) + 2 (h - kv) kh + 4 kv kh."""
    return 2 * kv * (w - kh) + 2 * (h - kv) * kh + 4 * kv * kh


def multiple_side(Y: dict, kh: int, kv: int) -> np.ndarray:
    """The coefficients of the four adjusted pairings that can differ from Y_DD, each
    distinct value once, concatenated (each region row-major):
      R_S, R_C            rows < kv, columns >= kh of Y_S*, Y_C* (independent of the
                          horizontal choice there);
      L_S, L_C            rows >= kv, columns < kh of Y_*S, Y_*C (independent of the
                          vertical choice);
      X_SS, X_SC, X_CS, X_CC   rows < kv, columns < kh of each pairing.
    Everywhere else every pairing equals Y_DD."""
    parts = [Y["SS"][:kv, kh:], Y["CS"][:kv, kh:], Y["SS"][kv:, :kh], Y["SC"][kv:, :kh]]
    parts += [Y[ab][:kv, :kh] for ab in MULTI_COMBOS]
    return np.concatenate([np.asarray(p).ravel() for p in parts])


def multiple_assemble(y_dd, side, w: int, h: int, kh: int, kv: int) -> dict:
    """Inverse of the layout: the full h x w block of every pairing from Y_DD and the
    block's side regions."""
    y_dd = np.asarray(y_dd, dtype=np.float64).reshape(h, w)
    side = np.asarray(side, dtype=np.float64)
    pos = 0

    def take(r, c):
        nonlocal pos
        v = side[pos:pos + r * c].reshape(r, c)
        pos += r * c
        return v

    R = {"S": take(kv, w - kh), "C": take(kv, w - kh)}
    L = {"S": take(h - kv, kh), "C": take(h - kv, kh)}
    out = {"DD": y_dd.copy()}
    for ab in MULTI_COMBOS:
        Y = y_dd.copy()
        Y[:kv, kh:] = R[ab[0]]
        Y[kv:, :kh] = L[ab[1]]
        Y[:kv, :kh] = take(kv, kh)
        out[ab] = Y
    return out


def multiple_blocks(x_flat, blocks, tfs):
    """FP64 "Multiple" forward of a packed block buffer: (Y_DD in the blocks' layout,
    the side buffer, side offsets).  Every transform a block uses must be a DCT-2 with no
    adjustment (K = 0) or a post-adjustment with K <= n/2.  Block i's side regions start at
    offsets[i] (floats; blocks in list order, each region rounded up to a multiple of 4);
    offsets[-1] is the total."""
    x_flat = np.asarray(x_flat)
    y = np.zeros(x_flat.shape[0], dtype=np.float64)

    def kq(t):
        kind = int(t.kind if not isinstance(t, dict) else t["kind"])
        if kind == KIND_NONE:
            return 0, None
        q = np.asarray(t.q if not isinstance(t, dict) else t["q"], dtype=np.float64)
        return q.shape[0], q

    for t in tfs:
        get = (lambda k: t[k]) if isinstance(t, dict) else (lambda k: getattr(t, k))
        kind = int(get("kind"))
        if int(get("core")) != 0 or kind not in (KIND_NONE, KIND_POST):
            raise ValueError("the Multiple forward needs DCT-2 cores with no adjustment or a post-adjustment")
        if kind == KIND_POST and 2 * np.asarray(get("q")).shape[0] > int(get("n")):
            raise ValueError("the Multiple forward needs K <= n/2")

    sizes = []
    for b in blocks:
        w, h = int(b["w"]), int(b["h"])
        kh, _ = kq(tfs[int(b["tf_h"])])
        kv, _ = kq(tfs[int(b["tf_v"])])
        s = multiple_side_size(w, h, kh, kv)
        sizes.append((s + 3) // 4 * 4)
    offsets = np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))]).astype(np.int64)
    side = np.zeros(int(offsets[-1]), dtype=np.float64)
    for i, b in enumerate(blocks):
        w, h, o = int(b["w"]), int(b["h"]), int(b["offset"])
        kh, qh = kq(tfs[int(b["tf_h"])])
        kv, qv = kq(tfs[int(b["tf_v"])])
        X = x_flat[o:o + w * h].astype(np.float64).reshape(h, w)
        Y = multiple_2d(X, qh, qv)
        y[o:o + w * h] = Y["DD"].ravel()
        s = multiple_side(Y, kh, kv)
        side[offsets[i]:offsets[i] + s.size] = s
    return y, side, offsets


__all__ += ["MULTI_COMBOS", "post_c8_from_s7", "multiple_1d", "multiple_2d", "multiple_side_size",
            "multiple_side", "multiple_assemble", "multiple_blocks"]


# --------------------------------------------------------------------------
# Blocks inside a frame.  The adjusted transforms apply to W x B and B x H regions of a
# frame (Section 2.2), so a codec holds its residual as a frame; the transform reads each
# block from its position there, and the reconstruction goes back to the same position.
# --------------------------------------------------------------------------

FRAME_BLOCK_FIELDS = ("x", "y", "w", "h", "tf_h", "tf_v")


def frame_coef_offsets(blocks) -> np.ndarray:
    """Packed coefficient offsets of frame blocks: block i's coefficients follow those of
    blocks 0..i-1 in list order, h x w row-major each."""
    sz = np.asarray(blocks["w"], dtype=np.int64) * np.asarray(blocks["h"], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)


def forward_frame(frame, blocks, tfs) -> np.ndarray:
    """Packed FP64 coefficients of the blocks of a 2-D residual frame (rows = frame lines)."""
    frame = np.asarray(frame)
    off = frame_coef_offsets(blocks)
    out = np.zeros(int(off[-1]), dtype=np.float64)
    mats = [tf_matrix(t) for t in tfs]
    for i, b in enumerate(blocks):
        x, y, w, h = int(b["x"]), int(b["y"]), int(b["w"]), int(b["h"])
        X = frame[y:y + h, x:x + w].astype(np.float64)
        out[off[i]:off[i + 1]] = forward_2d(X, mats[int(b["tf_h"])], mats[int(b["tf_v"])]).ravel()
    return out


def inverse_frame(coef, blocks, tfs, frame_shape, fill=0.0) -> np.ndarray:
    """FP64 reconstruction frame of packed coefficients: every block's inverse placed at its
    position; samples outside every block keep `fill`."""
    coef = np.asarray(coef, dtype=np.float64)
    off = frame_coef_offsets(blocks)
    out = np.full(frame_shape, fill, dtype=np.float64)
    mats = [tf_matrix(t) for t in tfs]
    for i, b in enumerate(blocks):
        x, y, w, h = int(b["x"]), int(b["y"]), int(b["w"]), int(b["h"])
        Y = coef[off[i]:off[i + 1]].reshape(h, w)
        out[y:y + h, x:x + w] = inverse_2d(Y, mats[int(b["tf_h"])], mats[int(b["tf_v"])])
    return out


def round_to_int16(x) -> np.ndarray:
    """Round half to even and saturate to the int16 range."""
    return np.clip(np.rint(np.asarray(x, dtype=np.float64)), -32768, 32767).astype(np.int16)


__all__ += ["FRAME_BLOCK_FIELDS", "frame_coef_offsets", "forward_frame", "inverse_frame", "round_to_int16"]
