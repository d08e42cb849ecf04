"""GPU fitting pieces: the coding-gain proxy kernel against the oracle, the fitter's
gradient against finite differences of its loss, and the Procrustes fixed point."""

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def test_proxy_kernel_matches_oracle():
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib
    rng = np.random.default_rng(0)
    nb, h, w = 3000, 8, 16
    Y = rng.standard_normal((nb, h, w)) * rng.uniform(0.5, 5.0, (1, h, w))
    y = torch.from_numpy(Y.astype(np.float32).ravel()).cuda()
    g = torch.zeros_like(y)
    work = torch.zeros(65 * h * w, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = adj.lib()
    _lib.check(lib.adj_coding_gain_proxy(y.data_ptr(), nb, h * w, work.data_ptr(), loss.data_ptr(), g.data_ptr(), None))
    torch.cuda.synchronize()
    L, G = O.proxy_loss(Y.astype(np.float32).astype(np.float64))
    assert abs(float(loss.item()) - L) <= 1e-12 * max(1.0, abs(L))
    assert np.abs(g.cpu().numpy() - G.ravel()).max() <= 1e-6 * np.abs(G).max()


def _fitter(kind, blocks=1024, **kw):
    from paper_2505_23618_gb300 import fit
    if kind == 1:
        cfg = fit.FitConfig(n=32, core=0, kind=1, parities=(0, 1, 0, 1), blocks=blocks, seed=3, **kw)
    else:
        cfg = fit.FitConfig(n=32, core=2, kind=2, k=8, blocks=blocks, seed=3, **kw)
    return fit.Fitter(cfg)


@pytest.mark.parametrize("kind", [1, 2])
def test_fitter_gradient_vs_finite_differences(kind):
    f = _fitter(kind, lam=0.5)
    rng = np.random.default_rng(kind)
    p0 = f.params() + rng.uniform(-0.05, 0.05, f.params().size)
    f.set_params(p0)
    _, _, _, g = f.loss_and_grad()
    sel = rng.choice(p0.size, min(10, p0.size), replace=False)
    fd = []
    h = 1e-2
    for j in sel:
        vals = []
        for s in (2, 1, -1, -2):
            p = p0.copy()
            p[j] += s * h
            f.set_params(p)
            vals.append(f.loss_and_grad()[0])
        fd.append((8 * (vals[1] - vals[2]) - (vals[0] - vals[3])) / (12 * h))
    f.set_params(p0)
    fd = np.array(fd)
    assert np.linalg.norm(g[sel] - fd) / np.linalg.norm(fd) <= 1e-4
    f.close()


def test_post_fit_procrustes_fixed_point():
    """With only the basis term on M = K rows, the unconstrained optimum over orthogonal Q
    is the orthogonal Procrustes solution Q = U V^T of D_K B_K^T, where the fit starts:
    its gradient vanishes and moving away raises the loss."""
    f = _fitter(2, lam=0.0, m=8, blocks=64)
    q0 = f.q()
    loss0, _, _, g = f.loss_and_grad()
    assert np.linalg.norm(g) < 1e-9
    p0 = f.params()
    f.set_params(p0 + 1e-3 * np.random.default_rng(1).standard_normal(p0.size))
    assert f.loss_and_grad()[0] > loss0
    # and the start matches the oracle's matrix of the same parameterisation
    D = O.dst7(32)
    B = O.dst2(32)
    u, _, vt = np.linalg.svd(D[:8] @ B[:8].T)
    assert np.abs(q0 - u @ vt).max() < 1e-10
    f.close()


def test_band_fit_reduces_loss():
    f = _fitter(1, lam=0.1, lr=0.02)
    first = f.loss_and_grad()[0]
    last = f.run(steps=40)
    assert last < first
    f.close()


@pytest.mark.parametrize("kind", [1, 2])
def test_eq2_fit(kind):
    """The paper's criterion (Eq. 2): the fitter's term equals the oracle's weighted error of
    the same H, its gradient agrees with central differences, and a short fit lowers it."""
    f = _fitter(kind, lam=0.0, eq2=True, blocks=64)
    rng = np.random.default_rng(10 + kind)
    p0 = f.params() + rng.uniform(-0.05, 0.05, f.params().size)
    f.set_params(p0)
    loss, basis, _, g = f.loss_and_grad()
    assert abs(basis - O.eq2_weighted_error(f.H(), O.dst7(32))) <= 1e-12 * max(1.0, basis)
    assert loss == pytest.approx(basis, rel=1e-12)
    sel = rng.choice(p0.size, min(8, p0.size), replace=False)
    fd = []
    for j in sel:
        vals = []
        for s in (1, -1):
            p = p0.copy()
            p[j] += s * 1e-5
            f.set_params(p)
            vals.append(f.loss_and_grad()[0])
        fd.append((vals[0] - vals[1]) / 2e-5)
    f.set_params(p0)
    assert np.linalg.norm(g[sel] - np.array(fd)) / np.linalg.norm(fd) <= 1e-6
    first = f.loss_and_grad()[0]
    assert f.run(steps=30) < first
    f.close()
