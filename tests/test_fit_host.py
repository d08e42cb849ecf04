"""The fitter's host-side FP64 model (band H and its angle gradient, the Cayley map, its inverse
and its gradient, the basis and Eq. 2 terms) agrees with the oracle, which is pinned on its
own.  No GPU: only the pure-numpy parts of fit.py are called."""

import math

import numpy as np
import pytest

import oracle as O
from paper_2505_23618_gb300 import fit, targets


@pytest.mark.parametrize("n,core,parities", [(8, 0, (0, 1)), (16, 3, (0, 1, 0)), (32, 2, (1, 0, 1, 0)),
                                             (64, 1, (0, 1) * 6)])
def test_band_model_and_angle_gradient(n, core, parities):
    rng = np.random.default_rng(n + core)
    n_ang = sum(len(O.layer_pairs(n, p)) for p in parities)
    th = rng.uniform(-0.6, 0.6, n_ang)
    H = fit.band_H(n, core, parities, th)
    assert np.allclose(H, O.adjusted_matrix(n, core, O.KIND_BAND, parities, th), atol=1e-13)
    dH = rng.standard_normal((n, n))
    assert np.allclose(fit.band_angle_grad(n, core, parities, th, dH),
                       O.grad_band_angles(n, core, parities, th, dH), atol=1e-11)


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_host_cores_are_the_oracles(n):
    for c in range(4):
        assert np.allclose(targets.core(n, c), O.core_matrix(n, c), atol=1e-13)
    assert np.allclose(targets.dst7(n), O.dst7(n), atol=1e-13)
    assert np.allclose(targets.dct8(n), O.dct8(n), atol=1e-13)


@pytest.mark.parametrize("k", [2, 5, 8, 16])
def test_cayley_map_gradient_and_inverse(k):
    rng = np.random.default_rng(k)
    w = rng.normal(0, 0.3, k * (k - 1) // 2)
    dg = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    Q = fit.cayley_q(w, k, dg)
    assert np.allclose(Q, O.cayley(w, k, dg), atol=1e-13)
    gq = rng.standard_normal((k, k))
    assert np.allclose(fit.cayley_grad(w, k, dg, gq), O.cayley_grad(w, k, gq, dg), atol=1e-11)
    # the start point of a post fit: an orthogonal matrix of either determinant maps back (one
    # of determinant -1 always has the eigenvalue -1, which the plain Cayley map cannot reach)
    q0 = np.linalg.qr(rng.standard_normal((k, k)))[0]
    for q in (q0, q0 * np.r_[-1.0, np.ones(k - 1)][:, None]):
        w0, dg0 = fit.cayley_init(q)
        assert np.linalg.det(dg0[:, None] * q) > 0
        assert np.allclose(fit.cayley_q(w0, k, dg0), q, atol=1e-10)


def test_basis_and_eq2_terms():
    """basis_term (both criteria) on a stand-in fitter object: value and dL/dH."""
    n, k = 16, 8
    rng = np.random.default_rng(7)

    class Stub:
        pass

    s = Stub()
    s.cfg = fit.FitConfig(n=n, core=0, kind=2, k=k, m=5)
    s.D = targets.dst7(n)
    q0 = np.linalg.qr(rng.standard_normal((k, k)))[0]
    s.w, s.dg = fit.cayley_init(q0)
    s.q = lambda: fit.cayley_q(s.w, k, s.dg)
    s.H = lambda: fit.Fitter.H(s)
    H = O.adjusted_matrix(n, O.CORE_DCT2, O.KIND_POST, Q=q0)
    val, dH = fit.Fitter.basis_term(s)
    assert math.isclose(val, np.sum((H[:5] - s.D[:5]) ** 2), rel_tol=1e-12)
    assert np.allclose(dH[:5], 2 * (H[:5] - s.D[:5])) and not dH[5:].any()
    s.cfg.eq2 = True
    val, dH = fit.Fitter.basis_term(s)
    assert math.isclose(val, O.eq2_weighted_error(H, s.D), rel_tol=1e-12)
    wts = np.exp(-math.log(100.0) / n * np.arange(n))[:, None]
    assert np.allclose(dH, 2 * wts * (H - s.D))


def test_basis_table_of_the_eq2_band_fit():
    """The basis-vector table (Fig. 3 in numbers) of the stored 16-point Eq. 2 fit (6-tap band
    before the DST-3): the fitted H is the oracle's adjusted matrix, every row is a unit vector
    (|h - d|^2 = 2 - 2 <h, d>), and the low-frequency rows the criterion weights most are far
    closer to the DST-7 than the high-frequency ones and than the core alone."""
    import json
    import os
    import numpy as np
    import oracle
    from paper_2505_23618_gb300 import fit
    path = os.path.join(os.path.dirname(fit.__file__), "params", "fitted_eq2.json")
    with open(path) as f:
        rec = json.load(f)["eq2_band6_dst3_16"]
    H = fit.band_H(16, 3, tuple(rec["parities"]), np.asarray(rec["angles"]))
    Ho = oracle.adjusted_matrix(16, 3, 1, rec["parities"], rec["angles"])
    assert np.abs(H - Ho).max() <= 1e-12
    rows = fit.basis_table(rec)
    assert [r["k"] for r in rows] == list(range(16))
    for r in rows:
        assert abs(r["dist"] ** 2 - (2 - 2 * r["inner"])) <= 1e-12
    low = [r["dist"] for r in rows[:8]]
    high = [r["dist"] for r in rows[10:]]
    assert max(low) < 0.06 < 0.15 < min(high)
    assert all(r["dist"] < r["core_dist"] for r in rows)
    assert "| 0 | 1.000 |" in fit.basis_table_markdown(rec)
