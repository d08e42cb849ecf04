"""The allocation-free forward entry point agrees with the plan-based one and the oracle.

adj_transform_fwd_uniform_noalloc serves callers that may not allocate device memory
while they process (an encoder that reserved its GPU memory at start-up, a plug-in
without an allocator).  It keeps its scratch in a static device array shared by all
calls, so consecutive calls with different sizes and transforms must each give the
same coefficients as adj_transform_fwd, within the per-block tolerance against the
FP64 oracle, and write nothing outside their blocks.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import REL_TOL

pytestmark = pytest.mark.gpu

MAX_BLOCKS = 131072  # ADJ_NOALLOC_MAX_BLOCKS


def _batch(rng, tf_h, tf_v, n_blocks):
    w, h = tf_h.n, tf_v.n
    data = synth.ar1_blocks(rng, n_blocks, h, w, 0.9, 0.8, 60.0, 1023).reshape(-1)
    blocks = np.zeros(n_blocks, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(n_blocks, dtype=np.int64) * w * h
    blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = w, h, 0, 1
    return data, blocks


def _noalloc(lib, tf_h, tf_v, x, y, n_blocks, stream=None):
    from paper_2505_23618_gb300 import _lib
    dh, dv = _lib._DescArray([tf_h]), _lib._DescArray([tf_v])
    return lib.adj_transform_fwd_uniform_noalloc(dh.arr, dv.arr, n_blocks, x.data_ptr(), y.data_ptr(), stream)


def _rel_errors(a, b, data, n):
    a = a.reshape(n, -1)
    b = b.reshape(n, -1)
    xn = np.linalg.norm(data.reshape(n, -1).astype(np.float64), axis=1)
    return np.linalg.norm(a - b, axis=1), xn


def _check_call(lib, rng, tf_h, tf_v, n):
    import torch
    import paper_2505_23618_gb300 as adj
    data, blocks = _batch(rng, tf_h, tf_v, n)
    x = torch.from_numpy(data).cuda()
    # one guard sample past the last block: the call must not write there
    y_new = torch.full((data.size + 16,), -1.0, device="cuda")
    y_ref = torch.zeros(data.size, device="cuda")
    rc = _noalloc(lib, tf_h, tf_v, x, y_new, n)
    assert rc == 0, lib.adj_last_error().decode()
    with adj.Plan([tf_h, tf_v]) as plan:
        plan.set_blocks(blocks, data.size)
        plan.fwd(x, y_ref)
    torch.cuda.synchronize()
    out = y_new.cpu().numpy().astype(np.float64)
    assert np.all(out[data.size:] == -1.0)
    a = out[:data.size]
    # against the plan-based forward (same kernel) and against the FP64 oracle
    err, xn = _rel_errors(a, y_ref.cpu().numpy().astype(np.float64), data, n)
    assert np.all(err <= REL_TOL * xn), float(np.max(err / np.maximum(xn, 1e-30)))
    ref = oracle.forward_blocks(data, blocks, [tf_h, tf_v])
    err, xn = _rel_errors(a, ref, data, n)
    assert np.all(err <= REL_TOL * xn), float(np.max(err / np.maximum(xn, 1e-30)))


def test_noalloc_matches_plan_forward_and_oracle_in_a_row():
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    lib = adj.lib()
    rng = np.random.default_rng(2024)
    calls = [
        # 64x32: 2 blocks per tile
        (synth.random_band(rng, 64, synth.CORE_DST3, [0, 1] * 6),
         synth.random_post(rng, 32, synth.CORE_DCT2, 16), 700),
        # 8x16: 32 blocks per tile, 3001 is not a multiple of it
        (synth.random_band(rng, 8, synth.CORE_DCT3, [1, 0, 1]),
         synth.random_post(rng, 16, synth.CORE_DST2, 5), 3001),
        # 4x4: 256 blocks per tile, the largest batch the static array takes
        (synth.random_band(rng, 4, synth.CORE_DST2, [0, 1]),
         synth.random_post(rng, 4, synth.CORE_DCT3, 3), MAX_BLOCKS),
        # 4x4 again, a count that leaves the last tile partly filled
        (synth.Tf(n=4, core=synth.CORE_DCT2),
         synth.random_band(rng, 4, synth.CORE_DST3, [1, 0, 1, 0]), MAX_BLOCKS - 77),
        # 64x16 with a 64-point K = 32 post block along the rows (applied over the whole tile,
        # from the transposed Q the call uploads), 4 blocks per tile, 517 not a multiple of it
        (synth.random_post(rng, 64, synth.CORE_DST2, 32),
         synth.random_post(rng, 16, synth.CORE_DCT2, 8), 517),
    ]
    for tf_h, tf_v, n in calls:
        _check_call(lib, rng, tf_h, tf_v, n)

    # sizes beyond the static scratch are rejected before any GPU work
    tf_h, tf_v = calls[0][0], calls[0][1]
    x = torch.zeros(16, dtype=torch.int16, device="cuda")
    y = torch.zeros(16, device="cuda")
    rc = _noalloc(lib, tf_h, tf_v, x, y, MAX_BLOCKS + 1)
    assert rc == _lib.ERR_CODE["ADJ_ERR_UNSUPPORTED_SIZE"]
    assert b"ADJ_NOALLOC_MAX_BLOCKS" in lib.adj_last_error()


def test_noalloc_refuses_stream_capture():
    """Its uploads read host memory that lives only for the call, so recording the call into
    a CUDA graph is refused (nothing is enqueued) and the capture itself stays valid."""
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib

    torch.cuda.set_device(0)
    lib = adj.lib()
    rng = np.random.default_rng(7)
    tf_h, tf_v = synth.Tf(n=8, core=synth.CORE_DCT2), synth.Tf(n=8, core=synth.CORE_DCT2)
    x = torch.zeros(64, dtype=torch.int16, device="cuda")
    y = torch.zeros(64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = _noalloc(lib, tf_h, tf_v, x, y, 1, stream=C_stream(s))
        y.add_(1.0)
    assert rc == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    assert b"CUDA graph" in lib.adj_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert float(y.sum()) == 64.0
    # outside capture the same call runs
    data, _ = _batch(rng, tf_h, tf_v, 1)
    x.copy_(torch.from_numpy(data))
    assert _noalloc(lib, tf_h, tf_v, x, y, 1) == 0
    torch.cuda.synchronize()


def C_stream(s):
    import ctypes
    return ctypes.c_void_p(s.cuda_stream)
