"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and compare
with the FP64 oracle block by block."""

from __future__ import annotations

import numpy as np

import oracle
import synth

# Per-block forward tolerance: |Y_gpu - Y_oracle|_2 <= REL_TOL * |X|_2 (FP32 path vs FP64).
REL_TOL = 1e-5
# Round trip: |X_hat - X|_inf <= RT_TOL.
RT_TOL = 1e-2


def run_gpu(wl, blocks=None, total=None, x=None, y_init=None):
    """Forward then inverse of a workload on cuda:0; returns (Y, X_hat) as float64 numpy."""
    import torch
    import paper_2505_23618_gb300 as adj
    blocks = wl.blocks if blocks is None else blocks
    total = wl.total if total is None else total
    data = wl.data if x is None else x
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(blocks, total)
        xd = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        y = torch.zeros(total, dtype=torch.float32, device="cuda") if y_init is None else y_init.clone()
        plan.fwd(xd, y, torch.cuda.current_stream())
        xr = torch.zeros(total, dtype=torch.float32, device="cuda")
        plan.inv(y, xr, torch.cuda.current_stream())
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64), xr.cpu().numpy().astype(np.float64)


def sub_workload(wl, idx):
    """The blocks idx of wl, repacked contiguously (for oracle checks of a sample)."""
    b = wl.blocks[idx]
    sz = b["w"].astype(np.int64) * b["h"]
    off = np.zeros(len(b), np.int64)
    off[1:] = np.cumsum(sz)[:-1]
    src = b["offset"][:, None]
    data = np.concatenate([wl.data[o:o + s] for o, s in zip(b["offset"], sz)]) if len(b) else np.zeros(0, np.int16)
    nb = b.copy()
    nb["offset"] = off
    return synth.Workload(wl.name + "-sample", nb, data, wl.tfs, wl.clip), src


def per_block_errors(y, ref, x, blocks):
    """(|y-ref|_2, |x|_2) per block, summed segment by segment."""
    errs = np.empty(len(blocks))
    norms = np.empty(len(blocks))
    for i, b in enumerate(blocks):
        s = slice(int(b["offset"]), int(b["offset"]) + int(b["w"]) * int(b["h"]))
        errs[i] = np.linalg.norm(y[s] - ref[s])
        norms[i] = np.linalg.norm(x[s].astype(np.float64))
    return errs, norms


def check_forward(y, wl, blocks=None):
    blocks = wl.blocks if blocks is None else blocks
    ref = oracle.forward_blocks(wl.data, blocks, wl.tfs)
    errs, norms = per_block_errors(y, ref, wl.data, blocks)
    bad = errs > REL_TOL * norms
    assert not bad.any(), (f"{bad.sum()} blocks over tolerance; worst ratio "
                           f"{np.max(errs / np.maximum(norms, 1e-300)):.3e}")
    return float(np.max(errs / np.maximum(norms, 1e-300)))


def check_inverse(y, xr, wl, blocks=None):
    """The GPU inverse of the GPU forward's FP32 coefficients y against the oracle's FP64
    inverse of the same y: |X_gpu - X_oracle|_2 <= REL_TOL * |y|_2 per block."""
    blocks = wl.blocks if blocks is None else blocks
    ref = oracle.inverse_blocks(y, blocks, wl.tfs)
    errs, norms = per_block_errors(xr, ref, y, blocks)
    bad = errs > REL_TOL * norms
    assert not bad.any(), (f"{bad.sum()} blocks over tolerance (inverse); worst ratio "
                           f"{np.max(errs / np.maximum(norms, 1e-300)):.3e}")
    return float(np.max(errs / np.maximum(norms, 1e-300)))


def check_roundtrip(xr, wl, blocks=None, tol=RT_TOL):
    blocks = wl.blocks if blocks is None else blocks
    err = 0.0
    for b in blocks:
        s = slice(int(b["offset"]), int(b["offset"]) + int(b["w"]) * int(b["h"]))
        err = max(err, float(np.abs(xr[s] - wl.data[s]).max()))
    assert err <= tol, f"round trip error {err}"
    return err
