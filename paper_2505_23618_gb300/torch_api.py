"""torch conveniences over a Plan: output allocation and stream plumbing only."""

from __future__ import annotations


def _torch():
    import torch
    return torch


def forward(plan, resid, out=None, stream=None):
    """int16 residuals (CUDA tensor, plan.total samples) -> FP32 coefficients."""
    torch = _torch()
    if resid.dtype != torch.int16 or not resid.is_cuda:
        raise TypeError("resid must be a CUDA int16 tensor")
    if out is None:
        out = torch.zeros(plan.total, dtype=torch.float32, device=resid.device)
    s = stream if stream is not None else torch.cuda.current_stream(resid.device)
    plan.fwd(resid, out, s)
    return out


def inverse(plan, coef, out=None, stream=None):
    """FP32 coefficients (CUDA tensor) -> FP32 reconstruction."""
    torch = _torch()
    if coef.dtype != torch.float32 or not coef.is_cuda:
        raise TypeError("coef must be a CUDA float32 tensor")
    if out is None:
        out = torch.zeros(plan.total, dtype=torch.float32, device=coef.device)
    s = stream if stream is not None else torch.cuda.current_stream(coef.device)
    plan.inv(coef, out, s)
    return out


def roundtrip(plan, resid, stream=None):
    y = forward(plan, resid, stream=stream)
    return y, inverse(plan, y, stream=stream)


def forward_multiple(plan, resid, side_offsets=None, stream=None):
    """Multiple forward (Section 2.3): int16 residuals -> (2-D DCT-2 coefficients, side
    regions of the four DST-7 / DCT-8 pairings, side offsets).  Prepares the plan's block
    list for this form unless ``side_offsets`` from an earlier preparation is given."""
    torch = _torch()
    if resid.dtype != torch.int16 or not resid.is_cuda:
        raise TypeError("resid must be a CUDA int16 tensor")
    if side_offsets is None:
        side_offsets = plan.prepare_multiple()
    y = torch.zeros(plan.total, dtype=torch.float32, device=resid.device)
    side = torch.zeros(max(4, int(side_offsets[-1])), dtype=torch.float32, device=resid.device)
    s = stream if stream is not None else torch.cuda.current_stream(resid.device)
    plan.fwd_multiple(resid, y, side, s)
    return y, side, side_offsets
