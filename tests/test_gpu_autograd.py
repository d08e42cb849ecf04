"""GPU: the forward of FP32 blocks (adj_transform_fwd_f32) and the autograd function over
the forward transform.  The FP32 forward of integer-valued input reproduces the int16 forward
bit for bit and matches the FP64 oracle on fractional input; autograd gradients of <G, Y> with
respect to the input and the parameters match the oracle's analytic gradients, and a Cayley
map computed in torch chains through them to the oracle's dL/dw."""

import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import REL_TOL
from test_gpu_bwd import REL, mixed_with_dense, oracle_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2505_23618_gb300 as adj
    adj.lib()
    torch.cuda.set_device(0)
    yield


def _covered(wl):
    c = np.zeros(wl.total, bool)
    for b in wl.blocks:
        c[int(b["offset"]):int(b["offset"]) + int(b["w"]) * int(b["h"])] = True
    return c


@pytest.mark.parametrize("seed,n", [(11, 40), (12, 333)])
def test_fwd_f32_integer_input_equals_int16_forward(seed, n):
    import torch
    import paper_2505_23618_gb300 as adj
    wl = mixed_with_dense(seed, n)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x16 = torch.from_numpy(wl.data).cuda()
        y16 = torch.zeros(wl.total, device="cuda")
        y32 = torch.zeros(wl.total, device="cuda")
        plan.fwd(x16, y16)
        plan.fwd_f32(x16.float(), y32)
        torch.cuda.synchronize()
    assert torch.equal(y16, y32)


def test_fwd_f32_fractional_input_matches_oracle():
    import torch
    import paper_2505_23618_gb300 as adj
    wl = mixed_with_dense(13, 200)
    x = (wl.data.astype(np.float64) + np.random.default_rng(13).uniform(-0.5, 0.5, wl.total)).astype(np.float32)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        y = torch.zeros(wl.total, device="cuda")
        plan.fwd_f32(torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        y = y.cpu().numpy().astype(np.float64)
    ref = O.forward_blocks(x.astype(np.float64), wl.blocks, wl.tfs)
    for b in wl.blocks:
        o, m = int(b["offset"]), int(b["w"]) * int(b["h"])
        nx = max(np.linalg.norm(x[o:o + m].astype(np.float64)), 1e-30)
        assert np.linalg.norm(y[o:o + m] - ref[o:o + m]) <= REL_TOL * nx


@pytest.mark.parametrize("x_fp32", [True, False])
def test_autograd_matches_oracle_gradients(x_fp32):
    import torch
    import paper_2505_23618_gb300 as adj
    wl = mixed_with_dense(14, 120)
    G = np.random.default_rng(114).standard_normal(wl.total)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        if x_fp32:
            x = x.float().requires_grad_(True)
        params = adj.param_vector(plan, device="cuda").requires_grad_(True)
        y = adj.adjusted_transform(x, params, plan)
        ref_y = torch.zeros(wl.total, device="cuda")
        plan.fwd(torch.from_numpy(wl.data).cuda(), ref_y)
        assert torch.equal(y.detach(), ref_y)
        (y.double() * torch.from_numpy(G).cuda()).sum().backward()
        torch.cuda.synchronize()
        gp = params.grad.cpu().numpy()
        lay = plan.param_layout()
        gx = x.grad.cpu().numpy().astype(np.float64) if x_fp32 else None
    rgx, rgp = oracle_grads(wl, G)
    if x_fp32:
        cov = _covered(wl)
        assert np.abs(gx[cov] - rgx[cov]).max() <= 1e-5 * np.abs(rgx).max()
    for i, ref in rgp.items():
        got = gp[lay[i]:lay[i + 1]]
        assert np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30) <= REL, (i, wl.tfs[i].kind)


def test_autograd_follows_new_parameters():
    """A changed parameter vector is uploaded before the forward: the output equals a plan
    built with those parameters."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.random_small(15, 80)
    rng = np.random.default_rng(15)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        p = adj.param_vector(plan).numpy()
        lay = plan.param_layout()
        tfs2 = []
        for i, t in enumerate(wl.tfs):
            if t.kind == synth.KIND_BAND:
                t = synth.Tf(n=t.n, core=t.core, kind=t.kind, parities=t.parities,
                             angles=t.angles + rng.uniform(-0.1, 0.1, t.angles.size))
                p[lay[i]:lay[i + 1]] = t.angles
            elif t.kind == synth.KIND_POST:
                t = synth.Tf(n=t.n, core=t.core, kind=t.kind, q=synth.haar_orthogonal(rng, t.q.shape[0]))
                p[lay[i]:lay[i + 1]] = t.q.ravel()
            tfs2.append(t)
        x = torch.from_numpy(wl.data).cuda()
        y = adj.adjusted_transform(x, torch.from_numpy(p).cuda(), plan)
        torch.cuda.synchronize()
    with adj.Plan(tfs2) as plan2:
        plan2.set_blocks(wl.blocks, wl.total)
        y2 = torch.zeros(wl.total, device="cuda")
        plan2.fwd(x, y2)
        torch.cuda.synchronize()
    assert torch.equal(y, y2)


def test_cayley_chain_through_torch_matches_oracle():
    """Q = D (I + W)^-1 (I - W) computed in torch (FP64) from w; dL/dw through torch's autograd
    and the GPU backward equals the oracle's cayley_grad of its analytic dL/dQ."""
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(16)
    K, n = 8, 16
    post = synth.random_post(rng, n, synth.CORE_DCT2, K)
    data = synth.ar1_blocks(rng, 64, n, n, 0.9, 0.9, 40.0, 255).reshape(-1)
    blocks = np.zeros(64, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(64) * n * n
    blocks["w"] = blocks["h"] = n
    wl = synth.Workload("cayley", blocks, data, [post], 255)
    G = rng.standard_normal(wl.total)
    w0 = rng.uniform(-0.3, 0.3, K * (K - 1) // 2)
    D = np.where(rng.random(K) < 0.5, -1.0, 1.0)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        w = torch.tensor(w0, dtype=torch.float64, requires_grad=True)
        iu = torch.triu_indices(K, K, 1)
        S = torch.zeros(K, K, dtype=torch.float64).index_put((iu[0], iu[1]), w)
        S = S - S.T
        I = torch.eye(K, dtype=torch.float64)
        Q = torch.diag(torch.from_numpy(D)) @ torch.linalg.solve(I + S, I - S)
        y = adj.adjusted_transform(torch.from_numpy(data).cuda(), Q.reshape(-1).cuda(), plan)
        (y.double() * torch.from_numpy(G).cuda()).sum().backward()
        gw = w.grad.numpy()
    Qo = O.cayley(w0, K, D)
    wl_o = synth.Workload("cayley", blocks, data, [synth.Tf(n=n, core=synth.CORE_DCT2, kind=synth.KIND_POST, q=Qo)], 255)
    _, rgp = oracle_grads(wl_o, G)
    ref = O.cayley_grad(w0, K, rgp[0].reshape(K, K), D)
    assert np.linalg.norm(gw - ref) / np.linalg.norm(ref) <= REL


def test_torch_api_rejects_short_or_wrong_buffers():
    """Buffers shorter than the plan's samples, non-contiguous ones and a parameter vector of the
    wrong length are refused on the host, before any launch."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.random_small(17, 20)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        with pytest.raises(ValueError):
            adj.forward(plan, x[: wl.total - 16])
        with pytest.raises(ValueError):
            adj.inverse(plan, torch.zeros(wl.total - 16, device="cuda"))
        with pytest.raises(ValueError):
            adj.forward(plan, x, out=torch.zeros(wl.total - 4, device="cuda"))
        with pytest.raises(ValueError):
            adj.forward(plan, torch.zeros((2, wl.total), dtype=torch.int16, device="cuda")[:, 0])
        with pytest.raises(TypeError):
            adj.forward(plan, x.float())
        p = adj.param_vector(plan, device="cuda")
        with pytest.raises(ValueError):
            adj.adjusted_transform(x, p[:-1], plan)
        y = adj.adjusted_transform(x, p, plan)     # the right sizes still work
        torch.cuda.synchronize()
        assert y.numel() == wl.total
