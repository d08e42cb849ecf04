"""The sparsity-promoting design aid (offline, host FP64): its DST family against closed-form
relations and scipy, its gradient against finite differences, the orthogonality of its steps,
and the paper's finding for the DST-7 (a narrow band before the DST-3)."""

import numpy as np
import pytest

from paper_2505_23618_gb300 import explore, targets


@pytest.mark.parametrize("t", [1, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_dst_family_orthonormal(t, n):
    T = explore.dst(t, n)
    assert np.abs(T @ T.T - np.eye(n)).max() < 1e-12


def test_dst_family_relations():
    sfft = pytest.importorskip("scipy.fft")
    for t in (1, 4):
        ref = sfft.dst(np.eye(16), type=t, norm="ortho", axis=0)
        assert np.abs(explore.dst(t, 16) - ref).max() < 1e-12
    assert np.abs(explore.dst(6, 16) - explore.dst(7, 16).T).max() < 1e-12     # DST-6 = DST-7^T
    assert np.abs(explore.dst(4, 16) - explore.dst(4, 16).T).max() < 1e-12     # DST-4 is symmetric
    assert np.abs(explore.dst(5, 16) - explore.dst(5, 16).T).max() < 1e-12     # so is DST-5


@pytest.mark.parametrize("side", ["pre", "post"])
def test_objective_gradient(side):
    rng = np.random.default_rng(3)
    n = 8
    B, D = targets.core(n, 3), explore.dst(7, n)
    X = np.linalg.qr(rng.standard_normal((n, n)))[0]
    _, G = explore.objective(X, B, D, side, mu=0.3)
    E = rng.standard_normal((n, n))
    h = 1e-6
    fd = (explore.objective(X + h * E, B, D, side, 0.3)[0] - explore.objective(X - h * E, B, D, side, 0.3)[0]) / (2 * h)
    assert abs(fd - np.sum(G * E)) <= 1e-6 * max(1.0, abs(fd))


def test_optimise_properties():
    n = 16
    B, D = targets.core(n, 0), explore.dst(7, n)
    X, f = explore.optimise(B, D, "pre", mu=0.0, steps=50)
    assert f < 1e-20                                   # the exact start is optimal without sparsity
    X0 = B.T @ D
    f0, _ = explore.objective(X0, B, D, "pre", 0.02)
    X, f = explore.optimise(B, D, "pre", mu=0.02, steps=300)
    assert f < f0 and np.abs(X.T @ X - np.eye(n)).max() < 1e-10


def test_dst7_wants_a_band_before_the_dst3():
    """Section 2.2: for the DST-7 the sparse choice is a band before the DST-3; the search
    finds a narrow band there and wider structures before the DCT-2 and DST-2."""
    n = 16
    D = explore.dst(7, n)
    res = {}
    for name in ("DST-3", "DCT-2", "DST-2"):
        X, _ = explore.optimise(targets.core(n, explore.CORES[name]), D, "pre", mu=0.02, steps=3000)
        res[name] = explore.sparsity(X)
    assert res["DST-3"][1] <= 3
    assert res["DST-3"][1] < res["DCT-2"][1] and res["DST-3"][1] < res["DST-2"][1]
