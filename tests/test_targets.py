"""The package's DST-7 / DCT-8 inputs for the dense reference transform match the
oracle's closed forms, and the Eq. 5 chessboard helper matches S C S."""

import numpy as np
import pytest

import oracle as O
from paper_2505_23618_gb300 import targets


@pytest.mark.parametrize("n", (4, 8, 16, 32, 64))
def test_targets_match_oracle(n):
    assert np.abs(targets.dst7(n) - O.dst7(n)).max() < 1e-14
    assert np.abs(targets.dct8(n) - O.dct8(n)).max() < 1e-14
    rng = np.random.default_rng(n)
    q = np.linalg.qr(rng.standard_normal((n // 2, n // 2)))[0]
    S = O.alt_sign(n // 2)
    assert np.abs(targets.chessboard(q) - S @ q @ S).max() < 1e-15
