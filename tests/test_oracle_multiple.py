"""Pins of the oracle's simultaneous DST-7 / DCT-8 adjustments (Section 2.3, Eq. 5).

The checks tie the oracle's "Multiple" functions to facts outside them: the DST-7 and
DCT-8 closed forms (at K = n the adjustment of the DCT-2 reproduces both exactly, the
DCT-8 one only through Eq. 5), Eq. 3 between independently written matrices, the
chessboard sign pattern the paper describes, the claim that coefficients outside the
first K lines are not changed, and a brute-force inverse of the side layout.
``test_planted_multiple_mistakes`` shows that plausible slips are caught.
"""

import numpy as np
import pytest

import oracle as O
import synth

SIZES = (4, 8, 16, 32, 64)


def exact_s7_q(N):
    """Q with diag(Q) T^(C2) = T^(S7) at K = N: Q = T^(S7) T^(C2)^T (orthogonal)."""
    return O.dst7(N) @ O.dct2(N).T


def haar(rng, K):
    return synth.haar_orthogonal(rng, K)


# --------------------------------------------------------------------------
# pin functions (reused by the planted-mistake test)
# --------------------------------------------------------------------------

def pin_exact(multiple_1d, N):
    """At K = N the DST-7 adjustment reproduces T^(S7) and Eq. 5 must give T^(C8)."""
    _, Hs, Hc = multiple_1d(N, exact_s7_q(N))
    return max(np.abs(Hs - O.dst7(N)).max(), np.abs(Hc - O.dct8(N)).max())


def pin_eq3(multiple_1d, N, Q):
    """Eq. 3 with Eq. 5: H_C = S H_S R, so |H_C - T^(C8)| = |H_S - T^(S7)| (Frobenius)."""
    _, Hs, Hc = multiple_1d(N, Q)
    S, R = O.alt_sign(N), O.reversal(N)
    e1 = np.abs(Hc - S @ Hs @ R).max()
    e2 = abs(np.linalg.norm(Hc - O.dct8(N)) - np.linalg.norm(Hs - O.dst7(N)))
    return max(e1, e2)


def pin_chessboard(c8_from_s7, Q):
    """Same magnitudes, signs flipped in a chessboard pattern."""
    Qc = c8_from_s7(Q)
    K = Q.shape[0]
    err = 0.0
    for i in range(K):
        for j in range(K):
            want = Q[i, j] if (i + j) % 2 == 0 else -Q[i, j]
            err = max(err, abs(Qc[i, j] - want))
    return err


def maxabs(a):
    a = np.asarray(a)
    return float(np.abs(a).max()) if a.size else 0.0


def pin_rows(multiple_1d, N, Q):
    """Section 2.3: the adjustment changes only the first K outputs; the other rows of both
    adjusted transforms are DCT-2 rows."""
    B, Hs, Hc = multiple_1d(N, Q)
    K = Q.shape[0]
    return max(maxabs(Hs[K:] - O.dct2(N)[K:]), maxabs(Hc[K:] - O.dct2(N)[K:]), maxabs(B - O.dct2(N)))


def pin_unchanged(multiple_2d, X, Qh, Qv):
    """Outside the first kv rows and kh columns every pairing equals the 2-D DCT-2, and the
    shared regions agree between pairings."""
    kh, kv = Qh.shape[0], Qv.shape[0]
    Y = multiple_2d(X, Qh, Qv)
    err = 0.0
    for ab in O.MULTI_COMBOS:
        err = max(err, maxabs(Y[ab][kv:, kh:] - Y["DD"][kv:, kh:]))
    err = max(err, maxabs(Y["SS"][:kv, kh:] - Y["SC"][:kv, kh:]),
              maxabs(Y["CS"][:kv, kh:] - Y["CC"][:kv, kh:]),
              maxabs(Y["SS"][kv:, :kh] - Y["CS"][kv:, :kh]),
              maxabs(Y["SC"][kv:, :kh] - Y["CC"][kv:, :kh]))
    return err


def pin_layout(side_fn, X, Qh, Qv):
    """The side regions, put back by a brute-force index walk, must rebuild every pairing."""
    h, w = X.shape
    kh, kv = Qh.shape[0], Qv.shape[0]
    Y = O.multiple_2d(X, Qh, Qv)
    side = side_fn(Y, kh, kv)
    err = 0.0
    for ab in O.MULTI_COMBOS:
        a, b = "SC".index(ab[0]), "SC".index(ab[1])
        Z = Y["DD"].copy()
        for r in range(h):
            for c in range(w):
                if r < kv and c >= kh:      # R_a
                    pos = a * kv * (w - kh) + r * (w - kh) + (c - kh)
                elif r >= kv and c < kh:    # L_b
                    pos = 2 * kv * (w - kh) + b * (h - kv) * kh + (r - kv) * kh + c
                elif r < kv and c < kh:     # X_ab
                    pos = 2 * kv * (w - kh) + 2 * (h - kv) * kh + (2 * a + b) * kv * kh + r * kh + c
                else:
                    continue
                Z[r, c] = side[pos]
        err = max(err, maxabs(Z - Y[ab]))
    return err


# --------------------------------------------------------------------------
# the pins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", SIZES)
def test_exact_adjustment_gives_dst7_and_dct8(N):
    assert pin_exact(O.multiple_1d, N) < 1e-12


@pytest.mark.parametrize("N,K", [(4, 2), (8, 4), (16, 8), (32, 8), (32, 16), (64, 8), (64, 32)])
def test_eq3_and_eq5(N, K):
    Q = haar(np.random.default_rng(N * 100 + K), K)
    assert pin_eq3(O.multiple_1d, N, Q) < 1e-12
    assert pin_rows(O.multiple_1d, N, Q) == 0.0
    # the K x K block alone: C^(C8) = diag(S_K Q S_K, I)
    _, _, Hc = O.multiple_1d(N, Q)
    C8 = O.post_matrix(N, O.post_c8_from_s7(Q))
    assert np.abs(Hc - C8 @ O.dct2(N)).max() < 1e-12


@pytest.mark.parametrize("K", [1, 2, 3, 8, 16])
def test_chessboard(K):
    assert pin_chessboard(O.post_c8_from_s7, haar(np.random.default_rng(K), K)) == 0.0


def test_no_adjustment():
    D, Hs, Hc = O.multiple_1d(16, None)
    assert np.array_equal(D, O.dct2(16)) and np.array_equal(Hs, D) and np.array_equal(Hc, D)


@pytest.mark.parametrize("w,h,kh,kv", [(32, 32, 8, 8), (64, 16, 8, 4), (8, 64, 2, 32), (4, 4, 2, 2),
                                       (16, 32, 0, 8), (32, 8, 16, 0), (64, 64, 32, 32)])
def test_changed_region_and_layout(w, h, kh, kv):
    rng = np.random.default_rng(w * h + kh)
    Qh = haar(rng, kh) if kh else np.zeros((0, 0))
    Qv = haar(rng, kv) if kv else np.zeros((0, 0))
    X = rng.standard_normal((h, w))
    assert pin_unchanged(O.multiple_2d, X, Qh, Qv) < 1e-12
    Y = O.multiple_2d(X, Qh, Qv)
    side = O.multiple_side(Y, kh, kv)
    assert side.size == O.multiple_side_size(w, h, kh, kv) == 2 * kv * w + 2 * h * kh
    assert pin_layout(O.multiple_side, X, Qh, Qv) == 0.0
    back = O.multiple_assemble(Y["DD"], side, w, h, kh, kv)
    for k in ("DD",) + O.MULTI_COMBOS:
        assert np.array_equal(back[k], Y[k])
    # each pairing against its own adjusted transform through the general 2-D path
    for ab in O.MULTI_COMBOS:
        qv = Qv if ab[0] == "S" else O.post_c8_from_s7(Qv)
        qh = Qh if ab[1] == "S" else O.post_c8_from_s7(Qh)
        Hv = O.adjusted_matrix(h, 0, O.KIND_POST, Q=qv) if kv else O.dct2(h)
        Hh = O.adjusted_matrix(w, 0, O.KIND_POST, Q=qh) if kh else O.dct2(w)
        assert maxabs(Y[ab] - O.forward_2d(X, Hh, Hv)) < 1e-12


def test_fraction_changed_at_k8():
    """With K = 8 at 32 and 64 points, under half of a block's coefficients change in each
    adjusted pairing (Section 2.3)."""
    for n in (32, 64):
        changed = 8 * n + (n - 8) * 8
        assert changed / (n * n) < 0.5


def test_multiple_blocks_layout():
    rng = np.random.default_rng(11)
    tfs = [synth.Tf(n=32, core=0, kind=synth.KIND_POST, q=haar(rng, 8)),
           synth.Tf(n=16, core=0, kind=synth.KIND_POST, q=haar(rng, 3)),
           synth.Tf(n=8, core=0)]
    blocks = np.zeros(3, dtype=synth.BLOCK_DTYPE)
    blocks["w"] = [32, 16, 8]
    blocks["h"] = [16, 8, 32]
    blocks["tf_h"] = [0, 1, 2]
    blocks["tf_v"] = [1, 2, 0]
    blocks["offset"] = [0, 512, 640]
    x = rng.integers(-300, 300, 896).astype(np.int16)
    y, side, off = O.multiple_blocks(x, blocks, tfs)
    sizes = [2 * 3 * 32 + 2 * 16 * 8, 2 * 0 * 16 + 2 * 8 * 3, 2 * 8 * 8 + 2 * 32 * 0]
    assert list(np.diff(off)) == [(s + 3) // 4 * 4 for s in sizes]
    b = blocks[1]
    X = x[512:640].astype(float).reshape(8, 16)
    Y = O.multiple_2d(X, tfs[1].q, None)
    assert np.array_equal(side[off[1]:off[1] + sizes[1]], O.multiple_side(Y, 3, 0))
    assert np.array_equal(y[512:640], Y["DD"].ravel())
    with pytest.raises(ValueError):
        O.multiple_blocks(x, blocks, [synth.Tf(n=32, core=2)] + tfs[1:])
    with pytest.raises(ValueError):
        O.multiple_blocks(x, blocks, [synth.Tf(n=32, core=0, kind=synth.KIND_POST, q=haar(rng, 17))] + tfs[1:])


# --------------------------------------------------------------------------
# planted mistakes: each slip must trip at least one pin
# --------------------------------------------------------------------------

def test_planted_multiple_mistakes():
    rng = np.random.default_rng(5)
    Q8 = haar(rng, 8)

    def no_flip(N, Q=None):          # forgets Eq. 5: DCT-8 adjustment = DST-7 one
        B, Hs, _ = O.multiple_1d(N, Q)
        return B, Hs, Hs.copy()

    def one_sided(N, Q=None):        # S C (no right S)
        B = O.dct2(N)
        C = O.post_matrix(N, Q)
        return B, C @ B, O.alt_sign(N) @ C @ B

    def transposed(N, Q=None):       # Q^T instead of Q
        B = O.dct2(N)
        C = O.post_matrix(N, np.asarray(Q).T)
        S = O.alt_sign(N)
        return B, C @ B, S @ C @ S @ B

    def bottom(N, Q=None):           # the block at the bottom-right
        B = O.dct2(N)
        K = Q.shape[0]
        C = np.eye(N)
        C[N - K:, N - K:] = Q
        S = O.alt_sign(N)
        return B, C @ B, S @ C @ S @ B

    for bad in (no_flip, one_sided, transposed, bottom):
        caught = pin_exact(bad, 16) > 1e-6 or pin_eq3(bad, 32, Q8) > 1e-6 or pin_rows(bad, 32, Q8) > 1e-6
        assert caught, bad.__name__

    assert pin_chessboard(lambda Q: Q.copy(), Q8) > 1e-3            # no sign flip
    assert pin_chessboard(lambda Q: -Q, Q8) > 1e-3                  # wrong pattern

    def r_from_wrong_pairing(Y, kh, kv):   # R_C taken from a DST-7 vertical pairing
        Z = dict(Y)
        Z["CS"] = Y["SC"]
        return O.multiple_side(Z, kh, kv)

    def regions_swapped(Y, kh, kv):        # L regions before R regions
        s = O.multiple_side(Y, kh, kv)
        nr = 2 * kv * (Y["DD"].shape[1] - kh)
        nl = 2 * (Y["DD"].shape[0] - kv) * kh
        return np.concatenate([s[nr:nr + nl], s[:nr], s[nr + nl:]])

    X = rng.standard_normal((16, 32))
    Qv = haar(rng, 4)
    for bad in (r_from_wrong_pairing, regions_swapped):
        assert pin_layout(bad, X, Q8, Qv) > 1e-6, bad.__name__
    assert pin_layout(O.multiple_side, X, Q8, Qv) == 0.0
