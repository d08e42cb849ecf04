"""Finite-difference checks of the GPU backward at the size of the two DST-7 fits (the
Givens parameterisation after Eq. 2 and the post block of Section 2.2): the 64-point
DCT-2 with a 24-tap band (12 single-parity layers, 378 angles) and the 64-point DST-2
with a 32 x 32 post block through the Cayley map (496 parameters), each applied in both
directions of 1024 AR(1) 64 x 64 blocks (rho 0.95, sigma 40).

The loss is L = sum_b <Y_b, R_b> with fixed random R, accumulated in FP64 from the FP32
coefficients of the GPU forward.  Central differences use the 4-point stencil
(8 (L(+h) - L(-h)) - (L(+2h) - L(-2h))) / 12h at h and h/2 with one Richardson step
(the stencil's error is O(h^4)); the step sizes are large enough that FP32 rounding of the
4 M coefficients stays below the 1e-4 bar.  24 sampled parameters per fit; the check is
norm-wise, |g - g_FD| <= 1e-4 |g_FD|."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FD_REL = 1e-4
N_BLOCKS = 1024
N_SAMPLE = 24


def _blocks(rng):
    data = synth.ar1_blocks(rng, N_BLOCKS, 64, 64, 0.95, 0.95, 40.0, 255).reshape(-1)
    blocks = np.zeros(N_BLOCKS, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(N_BLOCKS) * 4096
    blocks["w"] = blocks["h"] = 64
    return data, blocks


def _richardson(f, h):
    def stencil(s):
        return (8 * (f(s) - f(-s)) - (f(2 * s) - f(-2 * s))) / (12 * s)
    return (16 * stencil(h / 2) - stencil(h)) / 15


def test_band_angles_378_vs_finite_differences():
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(41)
    band = synth.random_band(rng, 64, synth.CORE_DCT2, [0, 1] * 6)
    assert band.angles.size == 378
    data, blocks = _blocks(rng)
    R = rng.standard_normal(data.size)
    x = torch.from_numpy(data).cuda()
    r = torch.from_numpy(R).cuda()
    with adj.Plan([band]) as plan:
        plan.set_blocks(blocks, data.size)
        gp = torch.zeros(plan.param_layout()[-1], device="cuda")
        plan.bwd(x, r.float(), None, gp)
        g = gp.cpu().numpy().astype(np.float64)
        assert g.size == 378

        def loss(ang):
            plan.update_params([synth.Tf(n=64, core=band.core, kind=1, parities=band.parities, angles=ang)])
            y = adj.forward(plan, x)
            return float((y.double() * r).sum())

        sel = rng.choice(378, N_SAMPLE, replace=False)
        fd = []
        for j in sel:
            def f(s, j=j):
                a = band.angles.copy()
                a[j] += s
                return loss(a)
            fd.append(_richardson(f, 0.04))
    fd = np.array(fd)
    err = np.linalg.norm(g[sel] - fd) / np.linalg.norm(fd)
    assert err <= FD_REL, err


def test_cayley_post_496_vs_finite_differences():
    """Q = D (I + W)^-1 (I - W) in torch (FP64) from the 496 entries of the skew W; dL/dw by
    torch autograd through the GPU backward, against central differences in w."""
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(42)
    K = 32
    data, blocks = _blocks(rng)
    R = rng.standard_normal(data.size)
    w0 = rng.uniform(-0.2, 0.2, K * (K - 1) // 2)
    assert w0.size == 496
    D = np.where(rng.random(K) < 0.5, -1.0, 1.0)
    iu = np.triu_indices(K, 1)

    def q_of(w):
        S = np.zeros((K, K))
        S[iu] = w
        S = S - S.T
        I = np.eye(K)
        return np.diag(D) @ np.linalg.solve(I + S, I - S)

    post = synth.Tf(n=64, core=synth.CORE_DST2, kind=synth.KIND_POST, q=q_of(w0))
    x = torch.from_numpy(data).cuda()
    r = torch.from_numpy(R).cuda()
    with adj.Plan([post]) as plan:
        plan.set_blocks(blocks, data.size)
        w = torch.tensor(w0, dtype=torch.float64, requires_grad=True)
        iu_t = torch.triu_indices(K, K, 1)
        S = torch.zeros(K, K, dtype=torch.float64).index_put((iu_t[0], iu_t[1]), w)
        S = S - S.T
        I = torch.eye(K, dtype=torch.float64)
        Q = torch.diag(torch.from_numpy(D)) @ torch.linalg.solve(I + S, I - S)
        y = adj.adjusted_transform(x, Q.reshape(-1).cuda(), plan)
        (y.double() * r).sum().backward()
        g = w.grad.numpy().copy()

        def loss(wv):
            plan.update_params([synth.Tf(n=64, core=post.core, kind=2, q=q_of(wv))])
            y = adj.forward(plan, x)
            return float((y.double() * r).sum())

        sel = rng.choice(496, N_SAMPLE, replace=False)
        fd = []
        for j in sel:
            def f(s, j=j):
                wv = w0.copy()
                wv[j] += s
                return loss(wv)
            fd.append(_richardson(f, 0.02))
    fd = np.array(fd)
    err = np.linalg.norm(g[sel] - fd) / np.linalg.norm(fd)
    assert err <= FD_REL, err
