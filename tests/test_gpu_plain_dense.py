"""GPU parity of the plain (unfused) form and of the dense reference transform kind."""

import numpy as np
import pytest

import synth
from gpu_util import REL_TOL, check_forward, check_roundtrip
from paper_2505_23618_gb300 import targets

pytestmark = pytest.mark.gpu


def run(wl, plain):
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y = torch.zeros(wl.total, device="cuda")
        xr = torch.zeros(wl.total, device="cuda")
        (plan.fwd_plain if plain else plan.fwd)(x, y)
        (plan.inv_plain if plain else plan.inv)(y, xr)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64), xr.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("make", [synth.blocks32_band, synth.blocks32_64_mixed, lambda: synth.random_small(3, 500),
                                  lambda: synth.random_small(4, 37)])
def test_plain_form_parity(make):
    wl = make()
    y, xr = run(wl, plain=True)
    check_forward(y, wl)
    check_roundtrip(xr, wl)
    yf, _ = run(wl, plain=False)
    # the two forms compute the same operations on the same data
    assert np.abs(y - yf).max() <= 1e-4 * max(1.0, np.abs(yf).max())


def dense_workload(seed, n_blocks):
    rng = np.random.default_rng(seed)
    tfs = []
    ids = {}
    for n in synth.SIZES:
        ids[("s7", n)] = len(tfs)
        tfs.append(synth.Tf(n=n, core=0, kind=synth.KIND_DENSE, q=targets.dst7(n)))
        ids[("c8", n)] = len(tfs)
        tfs.append(synth.Tf(n=n, core=0, kind=synth.KIND_DENSE, q=targets.dct8(n)))
    sizes = np.array(synth.SIZES)
    w = rng.choice(sizes, n_blocks)
    h = rng.choice(sizes, n_blocks)
    th = np.array([ids[("s7", int(a))] for a in w])
    tv = np.array([ids[("c8", int(a))] for a in h])
    blocks, data = synth._pack((w, h, th, tv), rng, synth._stats_c2, 1023)
    return synth.Workload("dense", blocks, data, tfs, 1023)


@pytest.mark.parametrize("plain", [False, True])
def test_dense_reference_transform(plain):
    wl = dense_workload(11, 400)
    y, xr = run(wl, plain)
    assert check_forward(y, wl) <= REL_TOL
    check_roundtrip(xr, wl)


def test_adjusted_vs_dense_context_blocks():
    """8K-workload-like blocks transformed by adjusted DST-3/DCT-2 pairs and by the exact
    DST-7 / DCT-8: both match the oracle on the same blocks."""
    wl = synth.uhd8k(frames=1, width=512, height=4320 - 64 * 60)
    y, xr = run(wl, plain=False)
    check_forward(y, wl)
    tfs = [synth.Tf(n=64, core=0, kind=synth.KIND_DENSE, q=targets.dst7(64)),
           synth.Tf(n=64, core=0, kind=synth.KIND_DENSE, q=targets.dct8(64)),
           synth.Tf(n=32, core=0, kind=synth.KIND_DENSE, q=targets.dct8(32))]
    wl2 = synth.Workload("c5-dense", wl.blocks, wl.data, tfs, wl.clip)
    y2, _ = run(wl2, plain=False)
    check_forward(y2, wl2)


def test_graph_replay_matches_direct_calls():
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib
    wl = synth.random_small(21, 700)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y, xr = adj.roundtrip(plan, x)
        yp = torch.zeros_like(y)
        plan.fwd_plain(x, yp)
        gy = torch.zeros_like(y)
        gx = torch.zeros_like(y)
        g = plan.graph(_lib.GRAPH_ROUNDTRIP, x, gy, gx)
        gp = plan.graph(_lib.GRAPH_FWD_PLAIN, x, torch.zeros_like(y))
        gpi_out = torch.zeros_like(y)
        gpi = plan.graph(_lib.GRAPH_INV_PLAIN, yp, gpi_out)
        for _ in range(3):
            g.launch()
            gpi.launch()
        torch.cuda.synchronize()
        assert torch.equal(gy, y) and torch.equal(gx, xr)
        assert float((gpi_out - x.float()).abs().max()) <= 1e-2
        g.close(), gp.close(), gpi.close()


def test_autotune_and_tuning_roundtrip(tmp_path):
    """The autotuner picks a tuning that keeps results identical; the cache replays it."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.uhd_mixed(frames=1, width=1280, height=720)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y0, xr0 = adj.roundtrip(plan, x)
        y = torch.zeros_like(y0)
        xr = torch.zeros_like(y0)
        cache = str(tmp_path / "tune.txt")
        t = plan.autotune(x, y, xr, cache_path=cache, max_evals=12)
        y1, xr1 = adj.roundtrip(plan, x)
        torch.cuda.synchronize()
        # tiling changes only which CTA transforms a block, not the arithmetic
        assert torch.equal(y1, y0) and torch.equal(xr1, xr0)
        plan.set_tuning({"cap_div": [1] * 25, "ctas_per_sm": 0, "ranges_per_sm": 1})
        assert plan.autotune(x, y, xr, cache_path=cache) == t
        with pytest.raises(adj.AdjError):
            plan.set_tuning({"cap_div": [3] * 25, "ctas_per_sm": 0, "ranges_per_sm": 1})
