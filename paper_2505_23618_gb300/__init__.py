"""GB300-native adjusted trigonometric transforms (Said, Egilmez & Chao).

Batched separable 2-D transforms of residual blocks whose 1-D passes are a fast
DCT-2/DCT-3/DST-2/DST-3 core with a band pre-adjustment or a top-left
post-adjustment (H = C B A, Eq. 1).  All arithmetic runs in the hand-written CUDA
library behind the C ABI of include/adjtx.h; this package only marshals arguments.
"""

from ._lib import (ADJ_OK, BLOCK_DTYPE, ERR_CODE, ERRORS, EXPORTED, LIB_PATH, AdjError,  # noqa: F401
                   Plan, check, lib, load)
from .torch_api import forward, forward_multiple, inverse, roundtrip  # noqa: F401

__all__ = ["Plan", "AdjError", "forward", "forward_multiple", "inverse", "roundtrip", "BLOCK_DTYPE", "lib",
           "LIB_PATH", "EXPORTED"]
