"""The allocation-free forward entry point agrees with the plan-based one.

adj_transform_fwd_uniform_noalloc serves callers that may not allocate device memory
while they process (an encoder that reserved its GPU memory at start-up, a plug-in
without an allocator).  It keeps its scratch in a static device array shared by all
calls, so two calls in a row with different sizes and transforms must each give the
same coefficients as adj_transform_fwd.
"""

import ctypes as C

import numpy as np
import pytest

import synth
from gpu_util import REL_TOL

pytestmark = pytest.mark.gpu


def _batch(rng, tf_h, tf_v, n_blocks):
    w, h = tf_h.n, tf_v.n
    data = synth.ar1_blocks(rng, n_blocks, h, w, 0.9, 0.8, 60.0, 1023).reshape(-1)
    blocks = np.zeros(n_blocks, dtype=synth.BLOCK_DTYPE)
    blocks["offset"] = np.arange(n_blocks, dtype=np.int64) * w * h
    blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = w, h, 0, 1
    return data, blocks


def _noalloc(lib, tf_h, tf_v, x, y, n_blocks):
    from paper_2505_23618_gb300 import _lib
    dh, dv = _lib._DescArray([tf_h]), _lib._DescArray([tf_v])
    return lib.adj_transform_fwd_uniform_noalloc(dh.arr, dv.arr, n_blocks, x.data_ptr(), y.data_ptr(), None)


def test_noalloc_matches_plan_forward_twice():
    import torch
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import _lib

    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    lib = adj.lib()
    rng = np.random.default_rng(2024)
    calls = [
        (synth.random_band(rng, 64, synth.CORE_DST3, [0, 1] * 6),
         synth.random_post(rng, 32, synth.CORE_DCT2, 16), 700),
        (synth.random_band(rng, 8, synth.CORE_DCT3, [1, 0, 1]),
         synth.random_post(rng, 16, synth.CORE_DST2, 5), 3001),
    ]
    for tf_h, tf_v, n in calls:
        data, blocks = _batch(rng, tf_h, tf_v, n)
        x = torch.from_numpy(data).cuda()
        y_new = torch.full((data.size,), -1.0, device="cuda")
        y_ref = torch.zeros(data.size, device="cuda")
        rc = _noalloc(lib, tf_h, tf_v, x, y_new, n)
        assert rc == 0, lib.adj_last_error().decode()
        with adj.Plan([tf_h, tf_v]) as plan:
            plan.set_blocks(blocks, data.size)
            plan.fwd(x, y_ref)
        torch.cuda.synchronize()
        a = y_new.cpu().numpy().astype(np.float64).reshape(n, -1)
        b = y_ref.cpu().numpy().astype(np.float64).reshape(n, -1)
        xn = np.linalg.norm(data.reshape(n, -1).astype(np.float64), axis=1)
        err = np.linalg.norm(a - b, axis=1)
        assert np.all(err <= REL_TOL * xn), float(np.max(err / np.maximum(xn, 1e-30)))

    # sizes beyond the static scratch are rejected before any GPU work
    tf_h, tf_v = calls[0][0], calls[0][1]
    x = torch.zeros(16, dtype=torch.int16, device="cuda")
    y = torch.zeros(16, device="cuda")
    rc = _noalloc(lib, tf_h, tf_v, x, y, 131072 + 1)
    assert rc == _lib.ERR_CODE["ADJ_ERR_UNSUPPORTED_SIZE"]
    assert b"ADJ_NOALLOC_MAX_BLOCKS" in lib.adj_last_error()
