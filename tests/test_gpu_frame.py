"""GPU parity of the frame entry points (blocks read from and written back to a frame)
against the FP64 oracle: forward per block |Y_gpu - Y_oracle|_2 <= 1e-5 |X|_2; FP32 inverse
per block within 1e-5 |X|_2 of the oracle's; the int16 inverse reproduces the residual frame
exactly; samples outside every block are never written."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import REL_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2505_23618_gb300 as adj
    adj.lib()
    torch.cuda.set_device(0)
    yield


def random_frame_case(seed, fw=200, fh=136, stride=216, fill=0.85):
    """Blocks of random sizes placed greedily on a 4 x 4 grid (some cells left empty), in
    random list order, with random transforms; x positions are often 4 mod 8."""
    rng = np.random.default_rng(seed)
    wl = synth.random_small(seed, 1)
    tfs = wl.tfs
    by_n = {}
    for i, t in enumerate(tfs):
        by_n.setdefault(t.n, []).append(i)
    taken = np.zeros((fh // 4, fw // 4), bool)
    rows = []
    for _ in range(4000):
        w, h = (int(v) for v in rng.choice(synth.SIZES, 2))
        x = int(rng.integers(0, (fw - w) // 4 + 1)) * 4 if w <= fw else -1
        y = int(rng.integers(0, (fh - h) // 4 + 1)) * 4 if h <= fh else -1
        if x < 0 or y < 0:
            continue
        cells = taken[y // 4:(y + h) // 4, x // 4:(x + w) // 4]
        if cells.any():
            continue
        cells[...] = True
        rows.append((x, y, w, h, int(rng.choice(by_n[w])), int(rng.choice(by_n[h]))))
        if taken.mean() > fill:
            break
    blocks = np.array(rows, dtype=synth.FRAME_BLOCK_DTYPE)
    blocks = blocks[rng.permutation(blocks.size)]
    frame = rng.integers(-1023, 1024, (fh, stride)).astype(np.int16)
    return frame, blocks, tfs, fw, fh, stride


def run_frame(frame, blocks, tfs, fw, fh, stride):
    import torch
    import paper_2505_23618_gb300 as adj
    with adj.Plan(tfs) as plan:
        plan.set_frame_blocks(blocks, fw, fh, stride)
        x = torch.from_numpy(frame).cuda()
        y = torch.zeros(max(4, plan.total), device="cuda")
        plan.fwd_frame(x, y)
        sentinel = 12345.0
        rf = torch.full(frame.shape, sentinel, device="cuda")
        plan.inv_frame(y, d_frame_f32=rf)
        ri = torch.full(frame.shape, -7777, dtype=torch.int16, device="cuda")
        plan.inv_frame(y, d_frame_i16=ri)
        torch.cuda.synchronize()
        return (y.cpu().numpy().astype(np.float64)[:plan.total], rf.cpu().numpy().astype(np.float64),
                ri.cpu().numpy(), sentinel)


def check(frame, blocks, tfs, y, rf, ri, sentinel):
    ref = oracle.forward_frame(frame, blocks, tfs)
    off = oracle.frame_coef_offsets(blocks)
    covered = np.zeros(frame.shape, bool)
    for i, b in enumerate(blocks):
        x0, y0, w, h = (int(b[f]) for f in ("x", "y", "w", "h"))
        X = frame[y0:y0 + h, x0:x0 + w].astype(np.float64)
        nx = max(np.linalg.norm(X), 1e-30)
        assert np.linalg.norm(y[off[i]:off[i + 1]] - ref[off[i]:off[i + 1]]) <= REL_TOL * nx, (i, w, h)
        assert np.linalg.norm(rf[y0:y0 + h, x0:x0 + w] - X) <= REL_TOL * nx + 1e-3, (i, w, h)
        covered[y0:y0 + h, x0:x0 + w] = True
    assert np.array_equal(ri[covered], frame[covered]), "int16 round trip is not exact"
    assert (rf[~covered] == sentinel).all() and (ri[~covered] == -7777).all(), "samples outside blocks were written"
    # the FP32 reconstruction against the oracle's inverse of the oracle's coefficients
    rec = oracle.inverse_frame(ref, blocks, tfs, frame.shape)
    assert np.abs(rf[covered] - rec[covered]).max() <= 1e-2


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_frame_matches_oracle(seed):
    frame, blocks, tfs, fw, fh, stride = random_frame_case(seed)
    y, rf, ri, sentinel = run_frame(frame, blocks, tfs, fw, fh, stride)
    check(frame, blocks, tfs, y, rf, ri, sentinel)


def test_frame_full_size_uhd_mixed():
    """A 3840x2160 frame tiled like the mixed UHD workload (62,151 blocks, every block its own core x
    adjustment per direction): the int16 round trip is exact everywhere, and sampled blocks
    match the oracle."""
    frame, blocks, tfs = synth.uhd_mixed_frame()
    fh, stride = frame.shape
    y, rf, ri, sentinel = run_frame(frame, blocks, tfs, 3840, fh, stride)
    assert np.array_equal(ri[:, :3840], frame[:, :3840])
    idx = np.sort(np.random.default_rng(0).choice(blocks.size, 800, replace=False))
    off = oracle.frame_coef_offsets(blocks)
    sub = blocks[idx]
    ref = oracle.forward_frame(frame, sub, tfs)
    soff = oracle.frame_coef_offsets(sub)
    for j, i in enumerate(idx):
        b = blocks[i]
        X = frame[int(b["y"]):int(b["y"]) + int(b["h"]), int(b["x"]):int(b["x"]) + int(b["w"])].astype(np.float64)
        assert np.linalg.norm(y[off[i]:off[i + 1]] - ref[soff[j]:soff[j + 1]]) <= REL_TOL * max(np.linalg.norm(X), 1e-30)


def test_frame_matches_packed_path():
    """The frame forward gives the packed forward's coefficients bit for bit (same kernel
    arithmetic), for the same blocks packed in list order."""
    import torch
    import paper_2505_23618_gb300 as adj
    frame, blocks, tfs, fw, fh, stride = random_frame_case(9)
    off = oracle.frame_coef_offsets(blocks)
    packed = np.zeros(blocks.size, dtype=synth.BLOCK_DTYPE)
    packed["offset"] = off[:-1]
    for f in ("w", "h", "tf_h", "tf_v"):
        packed[f] = blocks[f]
    data = np.concatenate([frame[int(b["y"]):int(b["y"]) + int(b["h"]), int(b["x"]):int(b["x"]) + int(b["w"])].ravel()
                           for b in blocks])
    with adj.Plan(tfs) as plan:
        plan.set_blocks(packed, int(off[-1]))
        yp = adj.forward(plan, torch.from_numpy(data).cuda())
        torch.cuda.synchronize()
    y, _, _, _ = run_frame(frame, blocks, tfs, fw, fh, stride)
    assert np.array_equal(y, yp.cpu().numpy().astype(np.float64))


def test_frame_errors():
    import torch
    import paper_2505_23618_gb300 as adj
    tfs = [synth.Tf(n=8, core=0), synth.Tf(n=4, core=1)]

    def blk(*rows):
        return np.array(list(rows), dtype=synth.FRAME_BLOCK_DTYPE)

    with adj.Plan(tfs) as plan:
        cases = [
            ((blk((0, 0, 8, 8, 0, 0), (4, 4, 8, 8, 0, 0)), 32, 32, 32), "ADJ_ERR_INVALID_ARG"),   # overlap
            ((blk((28, 0, 8, 8, 0, 0)), 32, 32, 32), "ADJ_ERR_INVALID_ARG"),                      # outside
            ((blk((2, 0, 8, 8, 0, 0)), 32, 32, 32), "ADJ_ERR_MISALIGNED"),                        # x not on the grid
            ((blk((0, 0, 8, 8, 0, 0)), 32, 32, 36), "ADJ_ERR_MISALIGNED"),                        # stride
            ((blk((0, 0, 8, 8, 0, 0)), 32, 32, 24), "ADJ_ERR_MISALIGNED"),                        # stride < width
            ((blk((0, 0, 8, 4, 0, 0)), 32, 32, 32), "ADJ_ERR_PARAM_MISMATCH"),                    # h vs transform
        ]
        for args, name in cases:
            with pytest.raises(adj.AdjError) as e:
                plan.set_frame_blocks(*args)
            assert e.value.name == name, (args, e.value.name)
        x = torch.zeros((32, 32), dtype=torch.int16, device="cuda")
        y = torch.zeros(64, device="cuda")
        out = torch.zeros((32, 32), device="cuda")
        plan.set_blocks(np.zeros(0, dtype=synth.BLOCK_DTYPE), 0)
        with pytest.raises(adj.AdjError) as e:            # packed block list
            plan.fwd_frame(x, y)
        assert e.value.name == "ADJ_ERR_INVALID_ARG"
        plan.set_frame_blocks(blk((8, 4, 8, 8, 0, 0)), 32, 32, 32)
        plan.fwd_frame(x, y)
        with pytest.raises(adj.AdjError) as e:            # two outputs
            plan.inv_frame(y, d_frame_f32=out, d_frame_i16=x)
        assert e.value.name == "ADJ_ERR_INVALID_ARG"
        with pytest.raises(adj.AdjError) as e:            # no output
            plan.inv_frame(y)
        assert e.value.name == "ADJ_ERR_INVALID_ARG"
        with pytest.raises(adj.AdjError) as e:            # the Multiple forward is packed only
            plan.prepare_multiple()
        assert e.value.name == "ADJ_ERR_INVALID_ARG"
        torch.cuda.synchronize()
