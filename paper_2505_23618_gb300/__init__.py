"""GB300-native adjusted trigonometric transforms (Said, Egilmez & Chao).

Batched separable 2-D transforms of residual blocks whose 1-D passes are a fast
DCT-2/DCT-3/DST-2/DST-3 core with a band pre-adjustment or a top-left
post-adjustment (H = C B A, Eq. 1).  All arithmetic runs in the hand-written CUDA
library behind the C ABI of include/adjtx.h; this package only marshals arguments.
"""

from ._lib import (ADJ_OK, BLOCK_DTYPE, ERR_CODE, ERRORS, EXPORTED, LIB_PATH, TILE_INFO_DTYPE,  # noqa: F401
                   AdjError, Plan, check, layout_preview, lib, load)
from .torch_api import (adjusted_transform, autograd_function, forward, forward_multiple, inverse,  # noqa: F401
                        param_vector, roundtrip)

__all__ = ["Plan", "AdjError", "forward", "forward_multiple", "inverse", "roundtrip", "adjusted_transform",
           "autograd_function", "param_vector", "AdjFn", "BLOCK_DTYPE", "TILE_INFO_DTYPE", "layout_preview", "lib",
           "LIB_PATH", "EXPORTED"]


def __getattr__(name):
    if name == "AdjFn":   # torch.autograd.Function, built on first use
        return autograd_function()
    raise AttributeError(name)
