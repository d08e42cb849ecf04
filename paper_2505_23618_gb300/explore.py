"""Sparsity-promoting search for adjustment structures, the design aid the paper describes
before choosing its sparse adjustments (Section 2.2): with C = I, minimise over orthogonal A

    mu * sum_ij A_ij^2 / (0.05 + |A_ij|)  +  sum_ij e^{-alpha i} (H_ij - D_ij)^2,   H = B A,

(alpha = ln(100)/N, the weights of Eq. 2), and likewise over C with A = I (H = C B), for each
fast core B (DCT-2, DCT-3, DST-2, DST-3) and each remaining DST as the target D.  How sparse
the optimised adjustment comes out tells which core suits which target: the paper picks a band
before the DST-3 and a top-left block after the DCT-2 for the DST-7.

This is an offline tool on N x N matrices (no per-block work): plain FP64 host arithmetic,
Riemannian gradient descent on the orthogonal group with a Cayley retraction and backtracking,
started from the exact adjustment.  The paper writes the sparsity term with unit weight; at
that weight every optimised adjustment here collapses to a signed permutation with a large
error, so the term carries a weight mu (default 0.02, where the errors stay small).

    python -m paper_2505_23618_gb300.explore --n 16 --out explore.json
"""

from __future__ import annotations

import json
import math

import numpy as np

from . import targets

CORES = {"DCT-2": 0, "DCT-3": 1, "DST-2": 2, "DST-3": 3}


def dst(kind: int, n: int) -> np.ndarray:
    """Orthonormal DST of type 1, 4, 5, 6, 7 or 8 (rows are basis vectors)."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    if kind == 1:
        return math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * (k + 1) * (m + 1) / (n + 1))
    if kind == 4:
        return math.sqrt(2.0 / n) * np.sin(np.pi * (2 * k + 1) * (2 * m + 1) / (4 * n))
    if kind == 5:
        return math.sqrt(4.0 / (2 * n + 1)) * np.sin(2 * np.pi * (k + 1) * (m + 1) / (2 * n + 1))
    if kind == 6:
        return math.sqrt(4.0 / (2 * n + 1)) * np.sin(np.pi * (k + 1) * (2 * m + 1) / (2 * n + 1))
    if kind == 7:
        return targets.dst7(n)
    if kind == 8:
        e = np.ones(n)
        e[-1] = 1.0 / math.sqrt(2.0)
        t = math.sqrt(4.0 / (2 * n - 1)) * np.sin(np.pi * (2 * k + 1) * (2 * m + 1) / (2 * (2 * n - 1)))
        return t * e[:, None] * e[None, :]
    raise ValueError(f"DST type {kind}")


TARGETS = {f"DST-{t}": t for t in (1, 4, 5, 6, 7, 8)}


def objective(X, B, D, side: str, mu: float = 1.0):
    """Value and gradient (w.r.t. X) of mu * sparsity(X) + weighted error of H, with
    H = B X (side 'pre', X = A) or H = X B (side 'post', X = C)."""
    n = X.shape[0]
    w = np.exp(-math.log(100.0) / n * np.arange(n))[:, None]
    H = B @ X if side == "pre" else X @ B
    E = H - D
    a = np.abs(X)
    val = mu * float(np.sum(X * X / (0.05 + a))) + float(np.sum(w * E * E))
    g_sp = X * (0.1 + a) / (0.05 + a) ** 2          # d/dx of x^2 / (0.05 + |x|)
    GH = 2.0 * w * E
    g_err = B.T @ GH if side == "pre" else GH @ B.T
    return val, mu * g_sp + g_err


def _cayley_step(X, S, t):
    """X (I + t/2 S)^{-1} (I - t/2 S) for a skew-symmetric S: stays orthogonal."""
    n = X.shape[0]
    I = np.eye(n)
    return X @ np.linalg.solve(I + 0.5 * t * S, I - 0.5 * t * S)


def optimise(B, D, side: str, mu: float = 1.0, steps: int = 2000, start: str = "exact", tol: float = 1e-12):
    """Riemannian gradient descent on O(N) from the exact adjustment (B^T D or D B^T), which
    has zero error, or from the identity; backtracking line search on the Cayley curve."""
    n = B.shape[0]
    if start == "exact":
        X = B.T @ D if side == "pre" else D @ B.T
    else:
        X = np.eye(n)
    f, G = objective(X, B, D, side, mu)
    t = 1.0
    for _ in range(steps):
        S = X.T @ G
        S = 0.5 * (S - S.T)                      # descent direction in the Lie algebra
        gn = float(np.sum(S * S))
        if gn < tol:
            break
        while t > 1e-12:
            Xn = _cayley_step(X, S, t)
            fn, Gn = objective(Xn, B, D, side, mu)
            if fn <= f - 1e-4 * t * gn:
                break
            t *= 0.5
        else:
            break
        X, f, G = Xn, fn, Gn
        t = min(1.0, 2.0 * t)
    return X, f


def sparsity(X, thr: float = 0.05):
    """Fraction of entries below thr in magnitude, the band half-width (largest |i - j| of an
    entry at or above thr), and the block size: the smallest K such that every entry at or
    above thr outside the top-left K x K block is on the diagonal (diag(Q, I) structure)."""
    big = np.abs(X) >= thr
    i, j = np.nonzero(big)
    band = int(np.max(np.abs(i - j))) if i.size else 0
    off = i != j
    block = int(max(i[off].max(), j[off].max()) + 1) if off.any() else 0
    return float(1.0 - big.mean()), band, block


def explore(n: int = 16, mu: float = 0.02, steps: int = 3000):
    rows = []
    for tname, t in TARGETS.items():
        D = dst(t, n)
        for cname, c in CORES.items():
            B = targets.core(n, c)
            for side in ("pre", "post"):
                X, f = optimise(B, D, side, mu, steps)
                H = B @ X if side == "pre" else X @ B
                w = np.exp(-math.log(100.0) / n * np.arange(n))[:, None]
                zeros, band, block = sparsity(X)
                rows.append({"target": tname, "core": cname, "side": side, "objective": f,
                             "weighted_error": float(np.sum(w * (H - D) ** 2)), "zero_fraction": zeros,
                             "band_half_width": band, "block_k": block, "orthogonality": float(np.abs(X.T @ X - np.eye(n)).max())})
    return rows


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Sparsity-promoting search for DST adjustments.")
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--mu", type=float, default=0.02,
                    help="weight of the sparsity term (at 1 every adjustment collapses to a signed permutation)")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default=None, help="JSON file for the results")
    a = ap.parse_args(argv)
    rows = explore(a.n, a.mu, a.steps)
    print(f"{'target':7s} {'core':6s} {'side':5s} {'zeros':>6s} {'band':>5s} {'block':>6s} {'w.error':>9s}")
    for r in rows:
        print(f"{r['target']:7s} {r['core']:6s} {r['side']:5s} {r['zero_fraction']:6.2f} "
              f"{r['band_half_width']:5d} {r['block_k']:6d} {r['weighted_error']:9.4f}")
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"n": a.n, "mu": a.mu, "steps": a.steps, "rows": rows}, f, indent=1)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
