"""torch conveniences over a Plan: output allocation and stream plumbing only."""

from __future__ import annotations


def _torch():
    import torch
    return torch


def _check(t, dtypes, plan, what):
    """A contiguous CUDA tensor of one of `dtypes` holding at least plan.total samples (the
    kernels read and write plan.total samples; a shorter buffer would be overrun)."""
    torch = _torch()
    if t.dtype not in dtypes or not t.is_cuda:
        names = " or ".join(str(d).replace("torch.", "") for d in dtypes)
        raise TypeError(f"{what} must be a CUDA {names} tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < plan.total:
        raise ValueError(f"{what} holds {t.numel()} samples, the plan's blocks need {plan.total}")


def forward(plan, resid, out=None, stream=None):
    """int16 residuals (CUDA tensor, plan.total samples) -> FP32 coefficients."""
    torch = _torch()
    _check(resid, (torch.int16,), plan, "resid")
    if out is None:
        out = torch.zeros(plan.total, dtype=torch.float32, device=resid.device)
    _check(out, (torch.float32,), plan, "out")
    s = stream if stream is not None else torch.cuda.current_stream(resid.device)
    plan.fwd(resid, out, s)
    return out


def inverse(plan, coef, out=None, stream=None):
    """FP32 coefficients (CUDA tensor) -> FP32 reconstruction."""
    torch = _torch()
    _check(coef, (torch.float32,), plan, "coef")
    if out is None:
        out = torch.zeros(plan.total, dtype=torch.float32, device=coef.device)
    _check(out, (torch.float32,), plan, "out")
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
    _check(resid, (torch.int16,), plan, "resid")
    if side_offsets is None:
        side_offsets = plan.prepare_multiple()
    y = torch.zeros(plan.total, dtype=torch.float32, device=resid.device)
    side = torch.zeros(max(4, int(side_offsets[-1])), dtype=torch.float32, device=resid.device)
    s = stream if stream is not None else torch.cuda.current_stream(resid.device)
    plan.fwd_multiple(resid, y, side, s)
    return y, side, side_offsets


# ---------------------------------------------------------------------------------------
# Autograd: the forward transform as a differentiable function of its input and of the
# adjustment parameters (the design of Section 2.2 fits these parameters, Eq. 2).
# ---------------------------------------------------------------------------------------

def _layout(plan):
    lay = getattr(plan, "_param_layout", None)
    if lay is None:
        lay = plan.param_layout()
        plan._param_layout = lay
    return lay


def _field(tf, name, default=None):
    return tf.get(name, default) if isinstance(tf, dict) else getattr(tf, name, default)


def param_vector(plan, dtype=None, device=None):
    """The plan's parameters in its gradient layout (adj_plan_param_layout): per transform the
    band angles, the K x K post block Q (row major) or the n x n dense matrix; nothing for a
    plain core.  Returns a 1-D tensor (FP64 by default, on `device`)."""
    import numpy as np
    torch = _torch()
    lay = _layout(plan)
    v = np.zeros(lay[-1], dtype=np.float64)
    for i, tf in enumerate(plan.tfs):
        kind = int(_field(tf, "kind", 0))
        if kind == 1:
            v[lay[i]:lay[i + 1]] = np.asarray(_field(tf, "angles"), dtype=np.float64)
        elif kind in (2, 3):
            v[lay[i]:lay[i + 1]] = np.asarray(_field(tf, "q"), dtype=np.float64).ravel()
    return torch.tensor(v, dtype=dtype or torch.float64, device=device)


def _set_params(plan, values):
    """Upload parameter values given in the gradient layout (host FP64 array); the structure of
    every transform (n, core, kind, layer parities, K) is kept."""
    import numpy as np
    lay = _layout(plan)
    tfs = []
    for i, tf in enumerate(plan.tfs):
        kind = int(_field(tf, "kind", 0))
        d = {"n": int(_field(tf, "n")), "core": int(_field(tf, "core")), "kind": kind,
             "parities": _field(tf, "parities", np.zeros(0))}
        seg = values[lay[i]:lay[i + 1]]
        if kind == 1:
            d["angles"] = seg.copy()
        elif kind in (2, 3):
            k = int(round(np.sqrt(seg.size)))
            d["q"] = seg.reshape(k, k).copy()
        tfs.append(d)
    plan.update_params(tfs)
    plan._param_values = values.copy()


def _make_autograd():
    torch = _torch()
    import numpy as np

    class _AdjFn(torch.autograd.Function):
        """Y = forward transform of x (int16 or FP32 blocks in the plan's packed layout) under the
        parameter vector `params` (gradient layout, see param_vector).  The parameters are uploaded
        to the plan when they differ from its current ones (post blocks must stay orthogonal to
        1e-6, e.g. through a Cayley map computed in torch).  Backward: adj_transform_bwd gives
        dL/dx (FP32 inputs) and dL/dparams (band angles, Q entries, dense entries)."""

        @staticmethod
        def forward(ctx, x, params, plan):
            _check(x, (torch.int16, torch.float32), plan, "x")
            if params.dim() != 1 or params.numel() != _layout(plan)[-1]:
                raise ValueError(f"params must be a vector of {_layout(plan)[-1]} entries (param_vector layout)")
            vals = params.detach().to("cpu", torch.float64).numpy()
            cur = getattr(plan, "_param_values", None)
            s = torch.cuda.current_stream(x.device)
            if cur is None or cur.shape != vals.shape or not np.array_equal(cur, vals):
                # the upload is not ordered after launches on a non-blocking stream: let the
                # plan's earlier launches on this stream finish before their tables change
                s.synchronize()
                _set_params(plan, vals)
            y = torch.zeros(plan.total, dtype=torch.float32, device=x.device)
            if x.dtype == torch.int16:
                plan.fwd(x, y, s)
            else:
                plan.fwd_f32(x, y, s)
            ctx.plan, ctx.vals, ctx.p_dtype = plan, vals, params.dtype
            ctx.save_for_backward(x)
            return y

        @staticmethod
        def backward(ctx, gy):
            (x,) = ctx.saved_tensors
            plan = ctx.plan
            if not np.array_equal(plan._param_values, ctx.vals):
                torch.cuda.current_stream(x.device).synchronize()
                _set_params(plan, ctx.vals)
            need_x, need_p = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            gx = torch.zeros(plan.total, dtype=torch.float32, device=x.device) if need_x else None
            n_grad = _layout(plan)[-1]
            gp = torch.zeros(max(1, n_grad), dtype=torch.float32, device=x.device) if need_p else None
            if need_x or need_p:
                plan.bwd(x.contiguous(), gy.contiguous().float(), gx, gp, torch.cuda.current_stream(x.device),
                         x_fp32=x.dtype == torch.float32)
            if gp is not None:
                gp = gp[:n_grad].to(ctx.p_dtype)
            return gx, gp, None

    return _AdjFn


_ADJFN = None


def autograd_function():
    """The torch.autograd.Function of the forward transform (built on first use, so that
    importing the package does not import torch)."""
    global _ADJFN
    if _ADJFN is None:
        _ADJFN = _make_autograd()
    return _ADJFN


def adjusted_transform(x, params, plan):
    """Differentiable forward transform: Y(x, params) for the plan's block list;
    ``AdjFn.apply(x, params, plan)`` with AdjFn = autograd_function()."""
    return autograd_function().apply(x, params, plan)


def __getattr__(name):
    if name == "AdjFn":
        return autograd_function()
    raise AttributeError(name)
