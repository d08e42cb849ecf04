"""GPU backward: input and parameter gradients against the FP64 oracle's analytic
gradients and against finite differences of the GPU forward."""

import numpy as np
import pytest

import oracle as O
import synth
from paper_2505_23618_gb300 import targets

pytestmark = pytest.mark.gpu

REL = 2e-5     # GPU (FP32) vs oracle (FP64) analytic gradients, norm-wise per transform
FD_REL = 1e-4  # GPU gradient vs central differences of the GPU forward, norm-wise


def oracle_grads(wl, G):
    """Per-transform gradients of L = <G, Y> (so dL/dY = G) from the oracle."""
    dH = {}
    gX = np.zeros(wl.total)
    mats = {i: O.tf_matrix(t) for i, t in enumerate(wl.tfs)}
    for b in wl.blocks:
        w, h, o = int(b["w"]), int(b["h"]), int(b["offset"])
        X = wl.data[o:o + w * h].astype(np.float64).reshape(h, w)
        Gb = G[o:o + w * h].reshape(h, w)
        gx, dHh, dHv = O.grad_2d(X, Gb, mats[int(b["tf_h"])], mats[int(b["tf_v"])])
        gX[o:o + w * h] = gx.ravel()
        dH[int(b["tf_h"])] = dH.get(int(b["tf_h"]), 0) + dHh
        dH[int(b["tf_v"])] = dH.get(int(b["tf_v"]), 0) + dHv
    out = {}
    for i, t in enumerate(wl.tfs):
        if i not in dH or t.kind == 0:
            continue
        if t.kind == 1:
            out[i] = O.grad_band_angles(t.n, t.core, t.parities, t.angles, dH[i])
        elif t.kind == 2:
            out[i] = O.grad_post_q(t.n, t.core, t.k, dH[i]).ravel()
        else:
            out[i] = dH[i].ravel()
    return gX, out


def gpu_grads(wl, G, x_fp32=False):
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        lay = plan.param_layout()
        x = torch.from_numpy(wl.data).cuda()
        if x_fp32:
            x = x.float()
        gy = torch.from_numpy(G.astype(np.float32)).cuda()
        gx = torch.zeros(wl.total, device="cuda")
        gp = torch.zeros(max(1, lay[-1]), device="cuda")
        plan.bwd(x, gy, gx, gp)
        gp2 = torch.zeros_like(gp)
        plan.bwd(x, gy, None, gp2)
        torch.cuda.synchronize()
        assert torch.equal(gp, gp2), "backward is not deterministic"
        gp = gp.cpu().numpy().astype(np.float64)
        return gx.cpu().numpy().astype(np.float64), {i: gp[lay[i]:lay[i + 1]] for i in range(len(wl.tfs))}


def mixed_with_dense(seed, n_blocks):
    wl = synth.random_small(seed, n_blocks)
    tfs = list(wl.tfs)
    # swap a few vertical transforms for dense ones (DCT-8) of the same size
    rng = np.random.default_rng(seed)
    dense_ids = {}
    for n in synth.SIZES:
        dense_ids[n] = len(tfs)
        tfs.append(synth.Tf(n=n, core=0, kind=synth.KIND_DENSE, q=targets.dct8(n)))
    blocks = wl.blocks.copy()
    pick = rng.random(blocks.size) < 0.2
    blocks["tf_v"][pick] = [dense_ids[int(h)] for h in blocks["h"][pick]]
    return synth.Workload(wl.name + "-dense", blocks, wl.data, tfs, wl.clip)


@pytest.mark.parametrize("seed,n,x_fp32", [(1, 60, False), (2, 300, True), (3, 17, False)])
def test_backward_matches_oracle(seed, n, x_fp32):
    wl = mixed_with_dense(seed, n)
    G = np.random.default_rng(seed + 100).standard_normal(wl.total)
    gx, gp = gpu_grads(wl, G, x_fp32)
    rgx, rgp = oracle_grads(wl, G)
    covered = np.zeros(wl.total, bool)
    for b in wl.blocks:
        covered[b["offset"]:b["offset"] + int(b["w"]) * int(b["h"])] = True
    assert np.abs(gx[covered] - rgx[covered]).max() <= 1e-5 * np.abs(rgx).max()
    for i, ref in rgp.items():
        err = np.linalg.norm(gp[i] - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= REL, (i, wl.tfs[i].kind, err)
    for i, t in enumerate(wl.tfs):
        if i not in rgp:
            assert not np.any(gp[i]), "transform without blocks has a nonzero gradient"


def test_backward_config_like_fit_blocks():
    """64x64 AR(1) blocks with one band transform (12 layers) in both directions and one
    post transform (K=32) in both directions: the two parameterisations of the fit."""
    rng = np.random.default_rng(4)
    band = synth.random_band(rng, 64, synth.CORE_DCT2, [0, 1] * 6)
    post = synth.random_post(rng, 64, synth.CORE_DST2, 32)
    n = 64
    data = synth.ar1_blocks(rng, n, 64, 64, 0.95, 0.95, 40.0, 255).reshape(-1)
    blocks = np.zeros(n, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(n) * 4096
    blocks["w"] = blocks["h"] = 64
    blocks["tf_h"] = blocks["tf_v"] = np.where(np.arange(n) < n // 2, 0, 1)
    wl = synth.Workload("fitlike", blocks, data, [band, post], 255)
    G = rng.standard_normal(wl.total)
    _, gp = gpu_grads(wl, G)
    _, rgp = oracle_grads(wl, G)
    for i in (0, 1):
        assert np.linalg.norm(gp[i] - rgp[i]) / np.linalg.norm(rgp[i]) <= REL


def test_backward_vs_finite_differences():
    """dL/dtheta and dL/dQ of the GPU backward agree with central differences of the GPU
    forward (loss accumulated in FP64 from FP32 coefficients), norm-wise within 1e-4."""
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(7)
    band = synth.random_band(rng, 32, synth.CORE_DST3, [0, 1, 0, 1])
    post = synth.random_post(rng, 16, synth.CORE_DCT2, 8)
    nb = 1024
    data = synth.ar1_blocks(rng, nb, 16, 32, 0.9, 0.9, 40.0, 255).reshape(-1)
    blocks = np.zeros(nb, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(nb) * 512
    blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = 32, 16, 0, 1
    R = rng.standard_normal(data.size)
    tfs = [band, post]
    x = torch.from_numpy(data).cuda()
    r = torch.from_numpy(R).cuda()
    with adj.Plan(tfs) as plan:
        plan.set_blocks(blocks, data.size)
        lay = plan.param_layout()
        gp = torch.zeros(lay[-1], device="cuda")
        plan.bwd(x, r.float(), None, gp)
        g = gp.cpu().numpy().astype(np.float64)

        def loss(ang, q):
            plan.update_params([synth.Tf(n=32, core=band.core, kind=1, parities=band.parities, angles=ang),
                                synth.Tf(n=16, core=post.core, kind=2, q=q)])
            y = adj.forward(plan, x)
            torch.cuda.synchronize()
            return float((y.double() * r).sum())

        sel = rng.choice(band.angles.size, 12, replace=False)
        fd_a = []
        for j in sel:
            hs = 1e-2
            vals = []
            for s in (2, 1, -1, -2):
                a = band.angles.copy()
                a[j] += s * hs
                vals.append(loss(a, post.q))
            fd_a.append((8 * (vals[1] - vals[2]) - (vals[0] - vals[3])) / (12 * hs))
        # Q lives on the orthogonal group: differentiate along a skew direction
        # Q(t) = Q expm(t S), dL/dt = <dL/dQ, Q S>
        fd_q, an_q = [], []
        gq = g[lay[1]:lay[2]].reshape(8, 8)
        for _ in range(4):
            S = rng.standard_normal((8, 8))
            S = S - S.T
            import scipy.linalg as sl
            vals = []
            hs = 1e-2
            for s in (2, 1, -1, -2):
                vals.append(loss(band.angles, post.q @ sl.expm(s * hs * S)))
            fd_q.append((8 * (vals[1] - vals[2]) - (vals[0] - vals[3])) / (12 * hs))
            an_q.append(float(np.sum(gq * (post.q @ S))))
    fd_a, an_a = np.array(fd_a), g[lay[0]:lay[1]][sel]
    assert np.linalg.norm(an_a - fd_a) / np.linalg.norm(fd_a) <= FD_REL
    fd_q, an_q = np.array(fd_q), np.array(an_q)
    assert np.linalg.norm(an_q - fd_q) / np.linalg.norm(fd_q) <= FD_REL
