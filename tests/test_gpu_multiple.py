"""GPU parity of the Multiple forward (Section 2.3, Eq. 5) against the FP64 oracle.

Per block: |Y_DD,gpu - Y_DD,oracle|_2 <= 1e-5 |X|_2 and the same bound for the block's
side regions (the distinct coefficients of the four DST-7 / DCT-8 pairings; each pairing
is orthogonal, so its coefficients have norm |X|_2 as well).  All calls go through the
C ABI.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import REL_TOL, sub_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2505_23618_gb300 as adj
    adj.lib()
    torch.cuda.set_device(0)
    yield


def multi_table(rng, ks=None):
    """Per size: a plain DCT-2 and DCT-2 + post-adjustments with several K <= n/2."""
    tfs, by_n = [], {}
    for n in synth.SIZES:
        by_n[n] = [len(tfs)]
        tfs.append(synth.Tf(n=n, core=0))
        choices = ks(n) if ks else sorted({1, max(1, n // 8), 3 if n >= 8 else 2, n // 2} - {0})
        for k in choices:
            if 1 <= k <= n // 2:
                by_n[n].append(len(tfs))
                tfs.append(synth.random_post(rng, n, synth.CORE_DCT2, k))
    return tfs, by_n


def make(seed, n_blocks, ks=None, shuffle=False):
    rng = np.random.default_rng(seed)
    tfs, by_n = multi_table(rng, ks)
    sizes = np.array(synth.SIZES)
    w = rng.choice(sizes, n_blocks)
    h = rng.choice(sizes, n_blocks)
    blocks = np.zeros(n_blocks, dtype=synth.BLOCK_DTYPE)
    off = 0
    for i in range(n_blocks):
        th = int(rng.choice(by_n[int(w[i])]))
        tv = int(rng.choice(by_n[int(h[i])]))
        blocks[i] = (off, w[i], h[i], th, tv)
        off += int(w[i] * h[i])
    data = np.zeros(off, np.int16)
    for b in blocks:
        ww, hh = int(b["w"]), int(b["h"])
        blk = synth.ar1_blocks(rng, 1, hh, ww, rng.uniform(0.6, 0.99), rng.uniform(0.6, 0.99),
                               float(np.exp(3 + rng.standard_normal())), 1023)
        data[b["offset"]:b["offset"] + ww * hh] = blk.ravel()
    if shuffle:
        blocks = blocks[rng.permutation(n_blocks)]
    return synth.Workload(f"multiple-{seed}", blocks, data, tfs, 1023)


def run_multiple(wl, tuning=None):
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        if tuning:
            plan.set_tuning(tuning)
        off = plan.prepare_multiple()
        x = torch.from_numpy(wl.data).cuda()
        y = torch.zeros(wl.total, device="cuda")
        side = torch.full((max(4, int(off[-1])),), float("nan"), device="cuda")
        plan.fwd_multiple(x, y, side)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64), side.cpu().numpy().astype(np.float64), off


def check(wl, y, side, off):
    ref_y, ref_side, ref_off = oracle.multiple_blocks(wl.data, wl.blocks, wl.tfs)
    assert np.array_equal(off, ref_off), "side offsets differ from the layout"
    worst = 0.0
    for i, b in enumerate(wl.blocks):
        s = slice(int(b["offset"]), int(b["offset"]) + int(b["w"]) * int(b["h"]))
        nx = np.linalg.norm(wl.data[s].astype(np.float64))
        e1 = np.linalg.norm(y[s] - ref_y[s])
        kh, kv = (int(getattr(wl.tfs[int(b[f])], "k", 0)) if wl.tfs[int(b[f])].kind == synth.KIND_POST else 0
                  for f in ("tf_h", "tf_v"))
        ss = slice(int(off[i]), int(off[i]) + oracle.multiple_side_size(int(b["w"]), int(b["h"]), kh, kv))
        assert not np.isnan(side[ss]).any(), "side region not written"
        e2 = np.linalg.norm(side[ss] - ref_side[ss]) if ss.stop > ss.start else 0.0
        if nx == 0:
            assert e1 == 0 and e2 == 0, "a zero block must give exact zeros"
            continue
        worst = max(worst, e1 / nx, e2 / (2 * nx))
        assert e1 <= REL_TOL * nx and e2 <= 2 * REL_TOL * nx, (i, int(b["w"]), int(b["h"]), e1 / nx, e2 / nx)
    return worst


@pytest.mark.parametrize("seed,n", [(1, 40), (2, 400), (3, 7)])
def test_multiple_matches_oracle(seed, n):
    wl = make(seed, n)
    y, side, off = run_multiple(wl)
    check(wl, y, side, off)


def test_multiple_caller_order_and_zero_blocks():
    wl = make(4, 120, shuffle=True)
    wl.data[wl.blocks["offset"][0]:wl.blocks["offset"][0] + int(wl.blocks["w"][0]) * int(wl.blocks["h"][0])] = 0
    y, side, off = run_multiple(wl)
    check(wl, y, side, off)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_multiple_small_k_everywhere(k):
    """One K at every size (K <= n/2), including K = 1 and the N = 4 case (KT = N)."""
    wl = make(10 + k, 150, ks=lambda n: [min(k, n // 2)])
    y, side, off = run_multiple(wl)
    check(wl, y, side, off)


def test_multiple_tile_capacity_and_tuning():
    """Many blocks of one class (several full tiles and a ragged tail), and a tuning that
    splits tiles and changes the grid: same results."""
    rng = np.random.default_rng(21)
    tfs = [synth.random_post(rng, 8, synth.CORE_DCT2, 4), synth.random_post(rng, 4, synth.CORE_DCT2, 2),
           synth.random_post(rng, 64, synth.CORE_DCT2, 32), synth.Tf(n=16, core=0)]
    cls = [(8, 4, 0, 1)] * 1000 + [(64, 16, 2, 3)] * 9 + [(4, 8, 1, 0)] * 77
    blocks = np.zeros(len(cls), dtype=synth.BLOCK_DTYPE)
    off = 0
    for i, (w, h, th, tv) in enumerate(cls):
        blocks[i] = (off, w, h, th, tv)
        off += w * h
    data = synth.ar1_blocks(rng, 1, 1, off, 0.9, 0.9, 60.0, 1023).reshape(-1)
    wl = synth.Workload("multiple-tiles", blocks, data, tfs, 1023)
    y, side, off_ = run_multiple(wl)
    check(wl, y, side, off_)
    tuning = {"cap_div": [4] * 25, "ctas_per_sm": 2, "ranges_per_sm": 3}
    y2, side2, _ = run_multiple(wl, tuning)
    check(wl, y2, side2, off_)


def test_multiple_agrees_with_fused_forward():
    """Each pairing rebuilt from Y_DD + side equals the fused forward with the post
    transforms Q (DST-7) or S Q S (DCT-8, Eq. 5) in each direction."""
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(7)
    qh, qv = synth.haar_orthogonal(rng, 8), synth.haar_orthogonal(rng, 4)
    nb, w, h = 200, 32, 16
    data = synth.ar1_blocks(rng, nb, h, w, 0.95, 0.9, 40.0, 1023).reshape(-1)
    blocks = np.zeros(nb, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(nb) * w * h
    blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = w, h, 0, 1
    tfs = [synth.Tf(n=w, core=0, kind=synth.KIND_POST, q=qh), synth.Tf(n=h, core=0, kind=synth.KIND_POST, q=qv)]
    wl = synth.Workload("multiple-vs-fused", blocks, data, tfs, 1023)
    y, side, off = run_multiple(wl)
    x = torch.from_numpy(data).cuda()
    qs = {"S": (qh, qv), "C": (oracle.post_c8_from_s7(qh), oracle.post_c8_from_s7(qv))}
    for ab in oracle.MULTI_COMBOS:
        t = [synth.Tf(n=w, core=0, kind=synth.KIND_POST, q=qs[ab[1]][0]),
             synth.Tf(n=h, core=0, kind=synth.KIND_POST, q=qs[ab[0]][1])]
        with adj.Plan(t) as plan:
            plan.set_blocks(blocks, wl.total)
            yf = adj.forward(plan, x)
            torch.cuda.synchronize()
            yf = yf.cpu().numpy().astype(np.float64)
        for i in range(0, nb, 13):
            o = i * w * h
            full = oracle.multiple_assemble(y[o:o + w * h], side[off[i]:off[i + 1]], w, h, 8, 4)[ab]
            ref = yf[o:o + w * h].reshape(h, w)
            assert np.linalg.norm(full - ref) <= 2e-6 * np.linalg.norm(ref), ab


def test_multiple_graph_replay_is_identical():
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib
    wl = make(31, 300)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        off = plan.prepare_multiple()
        x = torch.from_numpy(wl.data).cuda()
        y1 = torch.zeros(wl.total, device="cuda")
        s1 = torch.zeros(int(off[-1]), device="cuda")
        plan.fwd_multiple(x, y1, s1)
        y2, s2 = torch.zeros_like(y1), torch.zeros_like(s1)
        g = plan.graph(_lib.GRAPH_FWD_MULTIPLE, x, y2, s2)
        g.launch()
        g.launch()
        torch.cuda.synchronize()
        assert torch.equal(y1, y2) and torch.equal(s1, s2)
        g.close()


def test_multiple_errors():
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(3)
    code = adj.ERR_CODE
    bad_tfs = [[synth.random_band(rng, 8, 0, [0, 1])], [synth.Tf(n=8, core=2)],
               [synth.random_post(rng, 8, synth.CORE_DST3, 2)], [synth.Tf(n=8, core=0, kind=3, q=np.eye(8))]]
    blocks = np.zeros(1, dtype=synth.BLOCK_DTYPE)
    blocks[0] = (0, 8, 8, 0, 0)
    for tfs in bad_tfs:
        with adj.Plan(tfs) as plan:
            plan.set_blocks(blocks, 64)
            with pytest.raises(adj.AdjError) as e:
                plan.prepare_multiple()
            assert e.value.code == code["ADJ_ERR_INVALID_ARG"]
    with adj.Plan([synth.random_post(rng, 8, 0, 5)]) as plan:
        plan.set_blocks(blocks, 64)
        with pytest.raises(adj.AdjError) as e:
            plan.prepare_multiple()
        assert e.value.code == code["ADJ_ERR_UNSUPPORTED_SIZE"]
    with adj.Plan([synth.random_post(rng, 8, 0, 4)]) as plan:
        x = torch.zeros(64, dtype=torch.int16, device="cuda")
        y = torch.zeros(64, device="cuda")
        s = torch.zeros(256, device="cuda")
        with pytest.raises(adj.AdjError) as e:
            plan.fwd_multiple(x, y, s)
        assert e.value.code == code["ADJ_ERR_NO_BLOCKS"]
        plan.set_blocks(blocks, 64)
        with pytest.raises(adj.AdjError) as e:       # not prepared
            plan.fwd_multiple(x, y, s)
        assert e.value.code == code["ADJ_ERR_INVALID_ARG"]
        off = plan.prepare_multiple()
        assert int(off[-1]) == 2 * 4 * 8 + 2 * 8 * 4
        plan.fwd_multiple(x, y, s)
        plan.set_blocks(blocks, 64)                  # a new block list needs a new preparation
        with pytest.raises(adj.AdjError):
            plan.fwd_multiple(x, y, s)
        plan.prepare_multiple()
        with pytest.raises(adj.AdjError) as e:
            plan.fwd_multiple(x, y, s[1:])
        assert e.value.code == code["ADJ_ERR_MISALIGNED"]
        torch.cuda.synchronize()


def test_multiple_empty_and_unadjusted():
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan([synth.Tf(n=16, core=0)]) as plan:
        plan.set_blocks(np.zeros(0, dtype=synth.BLOCK_DTYPE), 0)
        assert list(plan.prepare_multiple()) == [0]
    # no adjustment anywhere: no side regions, Y_DD only
    wl = make(41, 60, ks=lambda n: [])
    y, side, off = run_multiple(wl)
    assert int(off[-1]) == 0
    check(wl, y, side, off)


def test_multiple_full_size_sampled():
    """The bench's workload (8 frames of 3840x2160, K = min(8, n/2)) in the bench's launch
    configuration, checked against the oracle on a sample of blocks."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.uhd_mixed_multiple()
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        off = plan.prepare_multiple()
        x = torch.from_numpy(wl.data).cuda()
        y = torch.zeros(wl.total, device="cuda")
        side = torch.zeros(int(off[-1]), device="cuda")
        plan.fwd_multiple(x, y, side)
        torch.cuda.synchronize()
        y = y.cpu().numpy().astype(np.float64)
        side = side.cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(0).choice(wl.blocks.size, 1500, replace=False)
    idx.sort()
    sub, src = sub_workload(wl, idx)
    ref_y, ref_side, ref_off = oracle.multiple_blocks(sub.data, sub.blocks, sub.tfs)
    for j, i in enumerate(idx):
        b = wl.blocks[i]
        n = int(b["w"]) * int(b["h"])
        o = int(b["offset"])
        nx = np.linalg.norm(wl.data[o:o + n].astype(np.float64))
        so = int(sub.blocks["offset"][j])
        assert np.linalg.norm(y[o:o + n] - ref_y[so:so + n]) <= REL_TOL * max(nx, 1e-30)
        ls = int(off[i + 1] - off[i])
        assert ls == int(ref_off[j + 1] - ref_off[j])
        assert np.linalg.norm(side[off[i]:off[i] + ls] - ref_side[ref_off[j]:ref_off[j] + ls]) <= 2 * REL_TOL * max(nx, 1e-30)
