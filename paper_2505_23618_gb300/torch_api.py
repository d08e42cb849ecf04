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
