"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each check ties the oracle to a closed form, a library routine, a relation the
paper states between independently written matrices, a published table or an
invariant.  ``test_planted_mistakes`` shows that plausible slips in the oracle
(dropped normalisation, transposed matrix, wrong rotation sign, reversed layer
order, flipped orientation) are caught by these checks.
"""

import math
import os

import numpy as np
import pytest

import oracle as O
import synth

SIZES = (4, 8, 16, 32, 64)
GOLD = os.path.join(os.path.dirname(__file__), "golden")
I = np.eye


def ortho_err(M):
    return np.abs(M.T @ M - I(M.shape[0])).max()


# --------------------------------------------------------------------------
# pin functions (reused by the planted-mistake test)
# --------------------------------------------------------------------------

def pin_scipy(fn, kind, typ, N):
    sfft = pytest.importorskip("scipy.fft")
    lib = getattr(sfft, kind)(np.eye(N), type=typ, norm="ortho", axis=0)
    return np.abs(fn(N) - lib).max()


def pin_relations(c2, c3, s2, s3, N):
    R, S = O.reversal(N), O.alt_sign(N)
    return max(np.abs(c3(N) - c2(N).T).max(),
               np.abs(s2(N) - R @ c2(N) @ S).max(),
               np.abs(s3(N) - S @ c2(N).T @ R).max())


def pin_eq3(s7, c8, N):
    return np.abs(c8(N) - O.alt_sign(N) @ s7(N) @ O.reversal(N)).max()


def pin_dst7_eigen(s7, N):
    L = 2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    L[N - 1, N - 1] = 1.0
    T = s7(N)
    lam = 2 - 2 * np.cos(np.pi * (2 * np.arange(N) + 1) / (2 * N + 1))
    return np.abs(L @ T.T - T.T * lam[None, :]).max()


def pin_layer_order(band):
    th0, th1 = 0.3, -0.7
    ang = np.zeros(3 + 2)           # N=6: even layer 3 pairs, odd layer 2 pairs
    ang[0] = th0                    # pair (0,1) of layer 0
    ang[3] = th1                    # pair (1,2) of layer 1
    A = band(6, [0, 1], ang)
    return abs(A[2, 0] - math.sin(th1) * math.sin(th0))


def pin_quarter_turn(layer, N):
    x = np.arange(1.0, N + 1)
    y = layer(N, 0, np.full(N // 2, np.pi / 2)) @ x
    want = np.empty(N)
    want[0::2] = -x[1::2]
    want[1::2] = x[0::2]
    return np.abs(y - want).max()


def pin_orientation(fwd, N_h=8, N_v=4):
    """A block whose rows are all equal only excites k_v = 0 with vertical DCT-2."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal(N_h)
    X = np.tile(x, (N_v, 1))
    Hh = O.adjusted_matrix(N_h, O.CORE_DST3, O.KIND_BAND, [0, 1],
                           rng.uniform(-1, 1, N_h // 2 + N_h // 2 - 1))
    Hv = O.dct2(N_v)
    Y = fwd(X, Hh, Hv)
    want = np.zeros_like(Y)
    want[0] = math.sqrt(N_v) * (Hh @ x)
    return np.abs(Y - want).max()


# --------------------------------------------------------------------------
# tests
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", SIZES)
def test_orthogonality(N):
    rng = np.random.default_rng(N)
    mats = [O.dct2(N), O.dct3(N), O.dst2(N), O.dst3(N), O.dst7(N), O.dct8(N), O.dct4(N),
            O.reversal(N), O.alt_sign(N)]
    par = [0, 1, 0, 1, 1, 0]
    cnt = sum(synth.n_pairs(N, p) for p in par)
    mats.append(O.band_matrix(N, par, rng.uniform(-np.pi, np.pi, cnt)))
    K = max(1, N // 2)
    Q = synth.haar_orthogonal(rng, K)
    mats.append(O.post_matrix(N, Q))
    for core in range(4):
        mats.append(O.adjusted_matrix(N, core, O.KIND_BAND, par, rng.uniform(-1, 1, cnt)))
        mats.append(O.adjusted_matrix(N, core, O.KIND_POST, Q=Q))
    for M in mats:
        assert ortho_err(M) < 1e-12


@pytest.mark.parametrize("N", SIZES)
def test_scipy_library_pins(N):
    assert pin_scipy(O.dct2, "dct", 2, N) < 1e-12
    assert pin_scipy(O.dct3, "dct", 3, N) < 1e-12
    assert pin_scipy(O.dct4, "dct", 4, N) < 1e-12
    assert pin_scipy(O.dst2, "dst", 2, N) < 1e-12
    assert pin_scipy(O.dst3, "dst", 3, N) < 1e-12


@pytest.mark.parametrize("N", SIZES)
def test_section21_relations(N):
    assert pin_relations(O.dct2, O.dct3, O.dst2, O.dst3, N) < 1e-12


@pytest.mark.parametrize("N", SIZES)
def test_eq3_dct8_is_flipped_dst7(N):
    assert pin_eq3(O.dst7, O.dct8, N) < 1e-12
    # the transposed (DST-6) reading of the DST-7 fails Eq. 3
    assert pin_eq3(lambda n: O.dst7(n).T, O.dct8, N) > 0.05


@pytest.mark.parametrize("N", SIZES)
def test_eq4_dct2_symmetry(N):
    S, R = O.alt_sign(N), O.reversal(N)
    assert np.abs(S @ O.dct2(N) - O.dct2(N) @ R).max() < 1e-12


@pytest.mark.parametrize("N,K", [(8, 4), (16, 8), (32, 8), (32, 16), (64, 32)])
def test_eq5_post_symmetry(N, K):
    """C^(C8) = S C^(S7) S turns a DST-7 post-adjustment into the DCT-8 one."""
    rng = np.random.default_rng(K)
    S, R = O.alt_sign(N), O.reversal(N)
    C7 = O.post_matrix(N, synth.haar_orthogonal(rng, K))
    C8 = S @ C7 @ S
    H7 = C7 @ O.dct2(N)
    H8 = C8 @ O.dct2(N)
    assert np.abs(H8 - S @ H7 @ R).max() < 1e-12
    # same approximation quality against the DCT-8 as against the DST-7
    e7 = np.linalg.norm(H7 - O.dst7(N))
    e8 = np.linalg.norm(H8 - O.dct8(N))
    assert abs(e7 - e8) < 1e-12
    # chessboard: same magnitudes, signs (-1)^(i+j)
    ij = np.add.outer(np.arange(N), np.arange(N))
    assert np.abs(C8 - C7 * (-1.0) ** ij).max() < 1e-15


@pytest.mark.parametrize("N", SIZES)
def test_dst7_eigenvectors(N):
    assert pin_dst7_eigen(O.dst7, N) < 1e-12


def test_golden_dct2_n4_radicals():
    a = math.sqrt(2 + math.sqrt(2)) / (2 * math.sqrt(2))
    b = math.sqrt(2 - math.sqrt(2)) / (2 * math.sqrt(2))
    rows = [eval(line, {"a": a, "b": b}) for line in open(os.path.join(GOLD, "dct2_n4_algebraic.txt"))
            if line.strip() and not line.startswith("#")]
    assert np.abs(O.dct2(4) - np.array(rows)).max() < 1e-15


def test_golden_hevc_dst7():
    tab = np.loadtxt(os.path.join(GOLD, "hevc_dst7_4x4.txt"))
    assert np.array_equal(np.rint(128 * O.dst7(4)), tab)


def test_dst3_approximates_dst7_low_frequency():
    """Section 2.2 pairs a band pre-adjustment with DST-3 to reach DST-7: row 0 is close."""
    for N in (16, 32, 64):
        assert O.dst3(N)[0] @ O.dst7(N)[0] > 0.99


@pytest.mark.parametrize("N", (2, 4, 8, 16, 32, 64))
def test_fast_core_matches_definition(N):
    assert np.abs(O.dct2_fast(np.eye(N)).T - O.dct2(N)).max() < 1e-12
    assert np.abs(O.dct4_fast(np.eye(N)).T - O.dct4(N)).max() < 1e-12


@pytest.mark.parametrize("N", SIZES)
def test_band_taps(N):
    """A K-tap band has at most K non-zeros per row (Section 2.2); L layers give 2L taps."""
    rng = np.random.default_rng(1)
    for L in (1, 2, 3, 4):
        par = [i % 2 for i in range(L)]
        cnt = sum(synth.n_pairs(N, p) for p in par)
        A = O.band_matrix(N, par, rng.uniform(0.1, 1.0, cnt))
        nnz = (np.abs(A) > 1e-14).sum(axis=1)
        assert nnz.max() == min(2 * L, N)
        assert np.all(np.abs(A[np.abs(np.subtract.outer(np.arange(N), np.arange(N))) > L]) < 1e-15)


def test_band_layer_order_and_sign():
    assert pin_layer_order(O.band_matrix) < 1e-15
    for N in SIZES:
        assert pin_quarter_turn(O.givens_layer, N) < 1e-13


def test_band_angle_counts():
    assert sum(synth.n_pairs(32, p) for p in [0, 1]) == 31
    assert sum(synth.n_pairs(64, p) for p in [0, 1] * 6) == 378
    with pytest.raises(ValueError):
        O.band_matrix(8, [0, 1], np.zeros(6))


@pytest.mark.parametrize("N,K", [(4, 2), (8, 8), (32, 8), (64, 32)])
def test_post_block_structure(N, K):
    """Only the first K outputs change (Section 2.3)."""
    rng = np.random.default_rng(3)
    Q = synth.haar_orthogonal(rng, K)
    for core in range(4):
        B = O.core_matrix(N, core)
        H = O.adjusted_matrix(N, core, O.KIND_POST, Q=Q)
        assert np.array_equal(H[K:], B[K:])
        assert np.abs(H[:K] - Q @ B[:K]).max() < 1e-14


def test_2d_orientation():
    assert pin_orientation(O.forward_2d) < 1e-12


def test_2d_roundtrip_parseval_zero():
    wl = synth.random_small(7, 40)
    Y = O.forward_blocks(wl.data, wl.blocks, wl.tfs)
    X = O.inverse_blocks(Y, wl.blocks, wl.tfs)
    assert np.abs(X - wl.data).max() < 1e-9
    for b in wl.blocks[:10]:
        s = slice(b["offset"], b["offset"] + int(b["w"]) * int(b["h"]))
        assert abs(np.linalg.norm(Y[s]) - np.linalg.norm(wl.data[s].astype(float))) < 1e-9
    Z = O.forward_blocks(np.zeros_like(wl.data), wl.blocks, wl.tfs)
    assert np.all(Z == 0.0)


@pytest.mark.parametrize("N_h,N_v", [(4, 4), (8, 4), (4, 8), (8, 8)])
def test_2d_brute_force_small(N_h, N_v):
    """Direct quadruple sum of the closed-form kernels at N = 4 and 8."""
    rng = np.random.default_rng(N_h * 10 + N_v)
    X = rng.integers(-50, 50, (N_v, N_h)).astype(float)
    ch, cv = 1, 2   # DCT-3 horizontally, DST-2 vertically, no adjustment
    Y = O.forward_2d(X, O.core_matrix(N_h, ch), O.core_matrix(N_v, cv))
    ref = np.zeros((N_v, N_h))
    for kv in range(N_v):
        dv = 1 / math.sqrt(2) if kv == N_v - 1 else 1.0
        for kh in range(N_h):
            acc = 0.0
            for r in range(N_v):
                for c in range(N_h):
                    ccol = 1 / math.sqrt(2) if c == 0 else 1.0
                    bh = ccol * math.sqrt(2 / N_h) * math.cos(math.pi * (2 * kh + 1) * c / (2 * N_h))
                    bv = dv * math.sqrt(2 / N_v) * math.sin(math.pi * (2 * r + 1) * (kv + 1) / (2 * N_v))
                    acc += bv * bh * X[r, c]
            ref[kv, kh] = acc
    assert np.abs(Y - ref).max() < 1e-10


def test_eq2_criterion():
    N = 16
    D = O.dst7(N)
    assert O.eq2_weighted_error(D, D) == 0.0
    E = np.zeros((N, N))
    E[0, 0] = 1.0
    E2 = np.zeros((N, N))
    E2[N - 1, 0] = 1.0
    assert O.eq2_weighted_error(D + E, D) == pytest.approx(1.0)
    # row N-1 weighs e^{-ln(100)(N-1)/N}
    assert O.eq2_weighted_error(D + E2, D) == pytest.approx(math.exp(-math.log(100) * (N - 1) / N))


def test_ar1_statistics():
    rng = np.random.default_rng(11)
    X = synth.ar1_blocks(rng, 4000, 16, 16, 0.9, 0.6, 1000.0, 32767).astype(float)
    r_row = np.mean(X[:, :, 1:] * X[:, :, :-1]) / np.mean(X * X)
    r_col = np.mean(X[:, 1:, :] * X[:, :-1, :]) / np.mean(X * X)
    assert abs(r_row - 0.9) < 0.01 and abs(r_col - 0.6) < 0.01
    assert abs(np.std(X) / 1000.0 - 1.0) < 0.02


def test_workload_layouts():
    wl = synth.blocks32_band()
    assert wl.total == 1024 * 1024 and wl.blocks.size == 1024
    wl3 = synth.uhd_mixed(frames=1, width=640, height=2160 - 64 * 27)
    off = wl3.blocks["offset"]
    sz = wl3.blocks["w"].astype(np.int64) * wl3.blocks["h"]
    assert np.all(off[1:] == off[:-1] + sz[:-1]) and off[-1] + sz[-1] == wl3.total
    assert int(sz.sum()) == 640 * (2160 - 64 * 27)
    assert np.all(off % 16 == 0)
    for b in wl3.blocks:
        assert wl3.tfs[b["tf_h"]].n == b["w"] and wl3.tfs[b["tf_v"]].n == b["h"]


def test_planted_mistakes():
    """Plausible slips in the oracle are caught by the pins above."""
    # dropped c_0 normalisation of the DCT-2
    def dct2_nonorm(N):
        T = O.dct2(N)
        T[0] *= math.sqrt(2)
        return T
    assert pin_scipy(dct2_nonorm, "dct", 2, 8) > 0.1
    # DST-2 written with the wrong index multiplying (2n+1)
    assert pin_relations(O.dct2, O.dct3, lambda N: O.dst3(N), O.dst3, 8) > 0.1
    # transposed DST-7
    assert pin_dst7_eigen(lambda N: O.dst7(N).T, 8) > 0.1
    # wrong DCT-8 phase
    assert pin_eq3(O.dst7, lambda N: O.dct8(N)[::-1], 8) > 0.1

    # rotation with a sign slip -> no longer orthogonal
    def layer_bad(N, parity, angles):
        G = O.givens_layer(N, parity, angles)
        for (i, j) in O.layer_pairs(N, parity):
            G[j, i] = -G[j, i]
        return G
    assert ortho_err(layer_bad(8, 0, np.full(4, 0.4))) > 0.1
    assert pin_quarter_turn(lambda N, p, a: O.givens_layer(N, p, a).T, 8) > 0.5

    # layers applied in the wrong order
    def band_reversed(N, parities, angles):
        A = np.eye(N)
        pos = 0
        for p in parities:
            cnt = len(O.layer_pairs(N, p))
            A = A @ O.givens_layer(N, p, angles[pos:pos + cnt])
            pos += cnt
        return A
    assert pin_layer_order(band_reversed) > 1e-3

    # 2-D transform with the horizontal / vertical roles swapped
    assert pin_orientation(lambda X, Hh, Hv: Hh @ X @ Hv.T, N_h=8, N_v=8) > 1e-3


# --------------------------------------------------------------------------
# blocks inside a frame
# --------------------------------------------------------------------------

def _frame_case(seed=0):
    rng = np.random.default_rng(seed)
    H, W = 48, 80
    frame = rng.integers(-300, 300, (H, W)).astype(np.int16)
    dt = np.dtype([("x", "<i4"), ("y", "<i4"), ("w", "<u2"), ("h", "<u2"), ("tf_h", "<u2"), ("tf_v", "<u2")])
    tfs = [synth.Tf(n=n, core=int(rng.integers(0, 4))) for n in (4, 8, 16, 32)]
    tfs += [synth.random_band(rng, 16, 3, [0, 1]), synth.random_post(rng, 32, 0, 8)]
    idx = {4: 0, 8: 1, 16: 2, 32: 3}
    rows = [(0, 0, 32, 16, 5, 2), (32, 0, 16, 16, 4, 4), (48, 4, 8, 8, 1, 1), (4, 16, 4, 32, 0, 3),
            (12, 20, 16, 4, 2, 0), (40, 24, 32, 8, 3, 1)]
    return frame, np.array(rows, dtype=dt), tfs


def test_frame_blocks_match_packed_blocks():
    """A frame block transforms exactly like the same samples packed on their own, and the
    inverse puts every block back at its position (round trip exact in FP64)."""
    frame, blocks, tfs = _frame_case()
    coef = O.forward_frame(frame, blocks, tfs)
    off = O.frame_coef_offsets(blocks)
    for i, b in enumerate(blocks):
        x, y, w, h = (int(b[f]) for f in ("x", "y", "w", "h"))
        packed = np.zeros(1, dtype=synth.BLOCK_DTYPE)
        packed[0] = (0, w, h, b["tf_h"], b["tf_v"])
        ref = O.forward_blocks(frame[y:y + h, x:x + w].ravel(), packed, tfs)
        assert np.array_equal(coef[off[i]:off[i + 1]], ref)
    rec = O.inverse_frame(coef, blocks, tfs, frame.shape, fill=np.nan)
    covered = ~np.isnan(rec)
    assert covered.sum() == int(off[-1])            # blocks do not overlap
    assert np.abs(rec[covered] - frame[covered]).max() < 1e-9
    assert np.array_equal(O.round_to_int16(rec[covered]), frame[covered])


def test_round_to_int16():
    x = np.array([0.5, 1.5, -0.5, -1.5, 2.4999, 40000.0, -40000.0, -2.5])
    assert list(O.round_to_int16(x)) == [0, 2, 0, -2, 2, 32767, -32768, -2]
