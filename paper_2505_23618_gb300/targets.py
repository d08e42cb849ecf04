"""The transforms the adjustments approximate (Section 2.2), as dense FP64 matrices.

They are inputs for the dense reference transform (kind ADJ_ADJ_DENSE), e.g. to time the
exact DST-7 / DCT-8 product beside the adjusted transforms.  Rows are basis vectors.
"""

from __future__ import annotations

import numpy as np


def dst7(n: int) -> np.ndarray:
    """DST-7: T[k, m] = sqrt(4 / (2n + 1)) sin(pi (2k + 1)(m + 1) / (2n + 1))."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    return np.sqrt(4.0 / (2 * n + 1)) * np.sin(np.pi * (2 * k + 1) * (m + 1) / (2 * n + 1))


def dct8(n: int) -> np.ndarray:
    """DCT-8, the flipped DST-7 of Eq. 3: T[k, m] = sqrt(4/(2n+1)) cos(pi (2k+1)(2m+1) / (4n+2))."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    return np.sqrt(4.0 / (2 * n + 1)) * np.cos(np.pi * (2 * k + 1) * (2 * m + 1) / (4 * n + 2))


def dense_tf(matrix: np.ndarray) -> dict:
    """A 1-D transform descriptor (dict form) applying `matrix` directly."""
    m = np.ascontiguousarray(matrix, dtype=np.float64)
    return {"n": m.shape[0], "core": 0, "kind": 3, "q": m}


def chessboard(q: np.ndarray) -> np.ndarray:
    """C^(C8) = S C^(S7) S (Eq. 5): the DCT-8 post-adjustment from the DST-7 one."""
    q = np.asarray(q, dtype=np.float64)
    s = (-1.0) ** np.arange(q.shape[0])
    return q * s[:, None] * s[None, :]


def core(n: int, kind: int) -> np.ndarray:
    """The fast cores of Section 2.1 as dense FP64 matrices (0 DCT-2, 1 DCT-3, 2 DST-2,
    3 DST-3), orthonormal; used by the fitter's host-side model of H."""
    k = np.arange(n)[:, None]
    m = np.arange(n)[None, :]
    c2 = np.sqrt(2.0 / n) * np.cos(np.pi * (2 * m + 1) * k / (2 * n))
    c2[0] /= np.sqrt(2.0)
    s2 = np.sqrt(2.0 / n) * np.sin(np.pi * (2 * m + 1) * (k + 1) / (2 * n))
    s2[n - 1] /= np.sqrt(2.0)
    return {0: c2, 1: c2.T.copy(), 2: s2, 3: s2.T.copy()}[int(kind)]
