"""GPU parity of the fused forward/inverse kernels against the FP64 oracle.

All calls go through the C ABI (paper_2505_23618_gb300.Plan).  Forward: per block
|Y_gpu - Y_oracle|_2 <= 1e-5 |X|_2; round trip: |X_hat - X|_inf <= 1e-2.
"""

import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import REL_TOL, RT_TOL, check_forward, check_inverse, check_roundtrip, run_gpu, sub_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2505_23618_gb300 as adj
    adj.lib()
    torch.cuda.set_device(0)
    yield


def make_workload(tfs, sizes, seed=0, clip=1023, order=None, gap=0):
    """Blocks of the given (w, h, tf_h, tf_v), AR(1) data, optional gaps / storage order."""
    rng = np.random.default_rng(seed)
    n = len(sizes)
    blocks = np.zeros(n, dtype=synth.BLOCK_DTYPE)
    off = 0
    for i, (w, h, th, tv) in enumerate(sizes):
        blocks[i] = (off, w, h, th, tv)
        off += w * h + gap
    total = off
    data = np.zeros(total, np.int16)
    for i, b in enumerate(blocks):
        w, h = int(b["w"]), int(b["h"])
        blk = synth.ar1_blocks(rng, 1, h, w, rng.uniform(0.6, 0.99), rng.uniform(0.6, 0.99),
                               float(np.exp(3 + rng.standard_normal())), clip)
        data[b["offset"]:b["offset"] + w * h] = blk.ravel()
    if order is not None:
        blocks = blocks[order]
    return synth.Workload("handmade", blocks, data, list(tfs), clip)


def full_check(wl):
    y, xr = run_gpu(wl)
    worst = check_forward(y, wl)
    check_inverse(y, xr, wl)
    rt = check_roundtrip(xr, wl)
    return worst, rt


def test_blocks32_band_full():
    worst, rt = full_check(synth.blocks32_band())
    assert worst < REL_TOL and rt < RT_TOL


def test_blocks32_64_mixed_full():
    worst, rt = full_check(synth.blocks32_64_mixed())
    assert worst < REL_TOL and rt < RT_TOL


@pytest.mark.parametrize("seed,n", [(1, 1), (2, 7), (3, 33), (4, 257), (5, 1001)])
def test_fuzz_mixed(seed, n):
    full_check(synth.random_small(seed, n))


@pytest.mark.parametrize("N", synth.SIZES)
@pytest.mark.parametrize("core", range(4))
@pytest.mark.parametrize("kind", range(3))
def test_every_core_kind_size_both_directions(N, core, kind):
    rng = np.random.default_rng(N * 100 + core * 10 + kind)
    if kind == 0:
        tf = synth.Tf(n=N, core=core)
    elif kind == 1:
        tf = synth.random_band(rng, N, core, [0, 1, 0, 1], -1.0, 1.0)
    else:
        tf = synth.random_post(rng, N, core, max(1, N // 2))
    other = {n: synth.Tf(n=n, core=int(rng.integers(4))) for n in synth.SIZES}
    tfs = [tf] + [other[n] for n in synth.SIZES]
    oi = {n: 1 + i for i, n in enumerate(synth.SIZES)}
    sizes = []
    for m in synth.SIZES:
        sizes += [(N, m, 0, oi[m])] * 3 + [(m, N, oi[m], 0)] * 3
    full_check(make_workload(tfs, sizes, seed=N + core + kind))


@pytest.mark.parametrize("N,K", [(8, 1), (8, 3), (8, 8), (16, 5), (32, 8), (32, 17), (64, 8), (64, 32),
                                 (64, 33), (64, 63), (64, 64), (4, 4), (4, 1)])
def test_post_block_sizes(N, K):
    rng = np.random.default_rng(K)
    tfs = [synth.random_post(rng, N, int(rng.integers(4)), K), synth.random_post(rng, N, 0, K)]
    sizes = [(N, N, 0, 1)] * 5 + [(N, N, 1, 0)] * 3
    full_check(make_workload(tfs, sizes, seed=K))


def test_tile_wide_inverse_post_blocks():
    """Inverse post blocks of padded size n / 2 on 16-, 32- and 64-sample lines run over the
    whole tile before the line pass (rows and columns); K below n / 2 pads to the same size.
    Every block shape that uses them, in full and partial tiles, against the oracle's inverse."""
    rng = np.random.default_rng(77)
    tfs = [synth.Tf(n=4, core=1), synth.random_post(rng, 8, 2, 3),
           synth.random_post(rng, 16, 0, 8), synth.random_post(rng, 16, 3, 5),
           synth.random_post(rng, 32, 1, 16), synth.random_post(rng, 32, 2, 11),
           synth.random_post(rng, 64, 0, 32), synth.random_post(rng, 64, 3, 20)]
    by_n = {4: [0], 8: [1], 16: [2, 3], 32: [4, 5], 64: [6, 7]}
    sizes = []
    for w in synth.SIZES:
        for h in synth.SIZES:
            for rep in range(int(rng.integers(1, 4)) * (3 if w * h <= 256 else 1)):
                sizes.append((w, h, int(rng.choice(by_n[w])), int(rng.choice(by_n[h]))))
    order = rng.permutation(len(sizes))
    worst, rt = full_check(make_workload(tfs, sizes, seed=77, order=order))
    assert worst < REL_TOL and rt < RT_TOL


@pytest.mark.parametrize("parities", [[], [1], [0], [1, 0, 1], [0, 1] * 32, [1] * 7])
def test_band_layer_structures(parities):
    rng = np.random.default_rng(len(parities))
    tfs = [synth.random_band(rng, n, int(rng.integers(4)), parities, -math.pi, math.pi) for n in synth.SIZES]
    sizes = [(w, h, i, j) for i, w in enumerate(synth.SIZES) for j, h in enumerate(synth.SIZES)]
    full_check(make_workload(tfs, sizes, seed=len(parities)))


@pytest.mark.parametrize("parities,lim", [([0, 1] * 32, 0.5), ([0, 1] * 32, 1.0), ([1, 0] * 6, 1.0),
                                          ([0, 1, 0, 1], 1.04)])
def test_band_angle_ranges_and_depths(parities, lim):
    """Deep bands (64 layers) and shallow ones with angles up to 0.5 and 1 rad, every size and
    a random core per size."""
    rng = np.random.default_rng(int(lim * 100) + len(parities))
    tfs = [synth.random_band(rng, n, int(rng.integers(4)), parities, -lim, lim) for n in synth.SIZES]
    sizes = [(w, h, i, j) for i, w in enumerate(synth.SIZES) for j, h in enumerate(synth.SIZES)] * 3
    full_check(make_workload(tfs, sizes, seed=len(parities)))


@pytest.mark.parametrize("w,h", [(4, 4), (8, 16), (16, 4), (32, 32), (64, 64), (64, 4), (4, 64)])
def test_tile_capacity_boundaries(w, h):
    cap = _tile_capacity(w, h)
    tfs = [synth.Tf(n=w, core=2), synth.Tf(n=h, core=3)]
    for n in (cap - 1, cap, cap + 1, 2 * cap + 3):
        if n < 1:
            continue
        full_check(make_workload(tfs, [(w, h, 0, 1)] * n, seed=n))


def _tile_capacity(w, h):
    # mirror of the planner's rule (4096 coefficients, at most 256 blocks per tile), used
    # only to pick boundary counts
    return min(4096 // (w * h), 256)


def test_unsorted_blocks_with_gaps_untouched_elsewhere():
    import torch
    rng = np.random.default_rng(9)
    tfs, ids = synth.mixed_tf_table(rng)
    sizes = []
    for _ in range(60):
        w, h = (int(x) for x in rng.choice(synth.SIZES, 2))
        sizes.append((w, h, ids[("h", w, int(rng.integers(4)), int(rng.integers(3)))],
                      ids[("v", h, int(rng.integers(4)), int(rng.integers(3)))]))
    order = rng.permutation(60)
    wl = make_workload(tfs, sizes, seed=3, order=order, gap=16)
    sentinel = torch.full((wl.total,), 7.25, dtype=torch.float32, device="cuda")
    y, xr = run_gpu(wl, y_init=sentinel)
    check_forward(y, wl)
    check_roundtrip(xr, wl)
    covered = np.zeros(wl.total, bool)
    for b in wl.blocks:
        covered[b["offset"]:b["offset"] + int(b["w"]) * int(b["h"])] = True
    assert np.all(y[~covered] == 7.25)


def test_zero_and_extreme_blocks():
    rng = np.random.default_rng(5)
    tfs, ids = synth.mixed_tf_table(rng)
    sizes = [(w, h, ids[("h", w, c, k)], ids[("v", h, (c + 1) % 4, (k + 1) % 3)])
             for w in synth.SIZES for h in synth.SIZES for c in range(4) for k in range(3)]
    wl = make_workload(tfs, sizes, seed=1)
    zero = np.zeros_like(wl.data)
    y, xr = run_gpu(wl, x=zero)
    assert np.all(y == 0.0) and np.all(xr == 0.0)
    ext = np.where(rng.random(wl.total) < 0.5, 32767, -32768).astype(np.int16)
    wl2 = synth.Workload("extreme", wl.blocks, ext, wl.tfs, 32768)
    y, xr = run_gpu(wl2)
    check_forward(y, wl2)
    # FP32 rounding scales with the magnitude: 1e-2 is the bound for 10-bit residuals
    # (|x| <= 1023); full-range int16 gets the same bound relative to its range.
    check_roundtrip(xr, wl2, tol=RT_TOL * 32768 / 1024)


def test_empty_block_list():
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan([synth.Tf(n=8, core=0)]) as plan:
        plan.set_blocks(np.zeros(0, synth.BLOCK_DTYPE), 64)
        x = torch.zeros(64, dtype=torch.int16, device="cuda")
        y = torch.full((64,), 3.0, device="cuda")
        plan.fwd(x, y)
        plan.inv(y, y.clone())
        torch.cuda.synchronize()
        assert torch.all(y == 3.0)
        assert plan.info()["n_tiles"] == 0


def test_repeated_launches_and_determinism():
    """The work counter resets itself: repeated launches give bit-identical output."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.random_small(77, 500)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        outs = []
        for _ in range(4):
            y = torch.zeros(wl.total, device="cuda")
            plan.fwd(x, y)
            outs.append(y)
        torch.cuda.synchronize()
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
    check_forward(outs[0].cpu().numpy().astype(np.float64), wl)


def test_host_entry_points_match_device_path():
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.random_small(8, 300)
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y_dev, xr_dev = adj.roundtrip(plan, x)
        torch.cuda.synchronize()
        h_in = torch.from_numpy(wl.data).pin_memory()
        h_y = torch.zeros(wl.total).pin_memory()
        h_x = torch.zeros(wl.total).pin_memory()
        plan.fwd_host(h_in, h_y)
        plan.inv_host(h_y, h_x)
        assert torch.equal(h_y, y_dev.cpu()) and torch.equal(h_x, xr_dev.cpu())


def test_host_path_chunked_matches_device_path():
    """Several host chunks (8.3 M samples, blocks listed out of storage order, gaps between
    blocks): the overlapped copy / kernel pipeline gives the device path's results bit for bit
    at every block sample."""
    import torch
    import paper_2505_23618_gb300 as adj
    wl = synth.uhd_mixed(frames=1)
    rng = np.random.default_rng(2)
    blocks = wl.blocks.copy()
    blocks = blocks[rng.random(blocks.size) < 0.8]           # leave gaps
    blocks = blocks[rng.permutation(blocks.size)]
    covered = np.zeros(wl.total, bool)
    for b in blocks:
        covered[b["offset"]:b["offset"] + int(b["w"]) * int(b["h"])] = True
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y_dev, xr_dev = adj.roundtrip(plan, x)
        torch.cuda.synchronize()
        h_in = torch.from_numpy(wl.data).pin_memory()
        h_y = torch.zeros(wl.total).pin_memory()
        h_x = torch.zeros(wl.total).pin_memory()
        for _ in range(2):
            plan.fwd_host(h_in, h_y)
            plan.inv_host(h_y, h_x)
        m = torch.from_numpy(covered)
        assert torch.equal(h_y[m], y_dev.cpu()[m]) and torch.equal(h_x[m], xr_dev.cpu()[m])
        plan.set_tuning({"cap_div": [2] * 25, "ctas_per_sm": 3, "ranges_per_sm": 2})
        h_y2 = torch.zeros(wl.total).pin_memory()
        plan.fwd_host(h_in, h_y2)
        assert torch.equal(h_y2[m], y_dev.cpu()[m])


def test_update_params_changes_result():
    import torch
    import paper_2505_23618_gb300 as adj
    rng = np.random.default_rng(4)
    wl = synth.blocks32_band()
    new = [synth.random_band(rng, 32, 0, [0, 1]), synth.random_band(rng, 32, 0, [0, 1])]
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        plan.update_params(new)
        x = torch.from_numpy(wl.data).cuda()
        y = adj.forward(plan, x)
        torch.cuda.synchronize()
        with pytest.raises(adj.AdjError) as e:
            plan.update_params([synth.random_band(rng, 32, 0, [0, 1, 0])] + new[1:])
        assert e.value.name == "ADJ_ERR_PARAM_MISMATCH"
    wl2 = synth.Workload("c1-new", wl.blocks, wl.data, new, 255)
    check_forward(y.cpu().numpy().astype(np.float64), wl2)


def test_set_blocks_and_launch_errors():
    import torch
    import paper_2505_23618_gb300 as adj
    tfs = [synth.Tf(n=8, core=0), synth.Tf(n=16, core=1)]
    B = synth.BLOCK_DTYPE

    def blocks(*rows):
        return np.array(list(rows), dtype=B)

    with adj.Plan(tfs) as plan:
        x = torch.zeros(4096, dtype=torch.int16, device="cuda")
        y = torch.zeros(4096, device="cuda")
        with pytest.raises(adj.AdjError) as e:
            plan.fwd(x, y)
        assert e.value.name == "ADJ_ERR_NO_BLOCKS"
        cases = [
            (blocks((0, 12, 8, 0, 0)), "ADJ_ERR_UNSUPPORTED_SIZE"),
            (blocks((0, 8, 8, 0, 5)), "ADJ_ERR_INVALID_ARG"),
            (blocks((0, 8, 16, 0, 0)), "ADJ_ERR_PARAM_MISMATCH"),
            (blocks((8, 8, 8, 0, 0)), "ADJ_ERR_MISALIGNED"),
            (blocks((0, 8, 8, 0, 0), (48, 8, 8, 0, 0)), "ADJ_ERR_INVALID_ARG"),
            (blocks((4064, 8, 8, 0, 0)), "ADJ_ERR_INVALID_ARG"),
            (blocks((-16, 8, 8, 0, 0)), "ADJ_ERR_MISALIGNED"),
        ]
        for bl, name in cases:
            with pytest.raises(adj.AdjError) as e:
                plan.set_blocks(bl, 4096)
            assert e.value.name == name, (bl, e.value)
        plan.set_blocks(blocks((0, 8, 8, 0, 0), (64, 16, 8, 1, 0)), 4096)
        with pytest.raises(adj.AdjError) as e:
            plan.fwd(x[1:], y)
        assert e.value.name == "ADJ_ERR_MISALIGNED"
        with pytest.raises(adj.AdjError) as e:
            plan.inv(y, y[2:])
        assert e.value.name == "ADJ_ERR_MISALIGNED"


# ---------------------------------------------------------------------------------
# Full-size configurations: every block is checked by properties that hold at any
# size (round trip, energy), a random sample of blocks against the oracle.
# ---------------------------------------------------------------------------------

def _full_size(wl, n_sample, seed):
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, wl.total)
        x = torch.from_numpy(wl.data).cuda()
        y, xr = adj.roundtrip(plan, x)
        torch.cuda.synchronize()
        xf = x.float()
        rt = float((xr - xf).abs().max())
        # Parseval per block: block energies of Y equal those of X (orthogonal transforms)
        idx = torch.from_numpy(np.repeat(np.arange(wl.blocks.size), (wl.blocks["w"].astype(np.int64) * wl.blocks["h"]))).cuda()
        ex = torch.zeros(wl.blocks.size, dtype=torch.float64, device="cuda").index_add_(0, idx, xf.double() ** 2)
        ey = torch.zeros(wl.blocks.size, dtype=torch.float64, device="cuda").index_add_(0, idx, y.double() ** 2)
        energy = float(((ey.sqrt() - ex.sqrt()).abs() / ex.sqrt().clamp_min(1e-30)).max())
        rng = np.random.default_rng(seed)
        pick = np.sort(rng.choice(wl.blocks.size, n_sample, replace=False))
        sub, _ = sub_workload(wl, pick)
        sizes = wl.blocks["w"][pick].astype(np.int64) * wl.blocks["h"][pick]
        sel = torch.from_numpy(np.concatenate([np.arange(o, o + s) for o, s in
                                               zip(wl.blocks["offset"][pick], sizes)])).cuda()
        ys = y[sel].cpu().numpy().astype(np.float64)
        del y, xr, x, xf
    assert rt <= RT_TOL, rt
    assert energy <= REL_TOL, energy
    return check_forward(ys, sub)


def test_uhd_mixed_full_size_sampled():
    assert _full_size(synth.uhd_mixed(), 3000, 3) <= REL_TOL


def test_uhd8k_full_size_sampled():
    assert _full_size(synth.uhd8k(), 1500, 5) <= REL_TOL


def _fitted_uhd8k_tfs():
    """The large-frame workload's transforms with the fitted parameters the benchmark times:
    horizontal DST-3 + 12-layer band (Section 2.2), vertical DCT-2 + post block with the
    DCT-8 block S Q S of Eq. 5 (K = 32 at 64 points, 16 at 32)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2505_23618_gb300", "params", "fitted.json")
    with open(path) as f:
        fit = json.load(f)
    b = fit["band_dst3_64"]
    h_tf = synth.Tf(n=64, core=synth.CORE_DST3, kind=synth.KIND_BAND,
                    parities=np.array(b["parities"], np.uint8), angles=np.array(b["angles"]))
    v_tfs = {}
    for n in (64, 32):
        p = fit[f"post_dct2_{n}"]
        q7, q8 = np.array(p["q"]), np.array(p["q_dct8"])
        # the stored DCT-8 block is the DST-7 one conjugated by the alternating signs (Eq. 5)
        assert np.abs(q8 - oracle.post_c8_from_s7(q7)).max() <= 1e-12
        v_tfs[n] = synth.Tf(n=n, core=synth.CORE_DCT2, kind=synth.KIND_POST, q=q8)
    return h_tf, v_tfs


def test_uhd8k_fitted_parameters_full_size_sampled():
    """The 16-frame 8K workload with the fitted parameters of the benchmark: round trip and
    per-block energy on every block, 1500 sampled blocks against the oracle."""
    h_tf, v_tfs = _fitted_uhd8k_tfs()
    assert h_tf.angles.size == 378
    assert _full_size(synth.uhd8k(h_tf=h_tf, v_tfs=v_tfs), 1500, 55) <= REL_TOL
