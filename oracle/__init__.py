"""FP64 CPU oracle for the adjusted 2-D transforms (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA library and its Python binding
never import it, and it imports nothing from them.
"""

from .adjtx_oracle import *  # noqa: F401,F403
from .adjtx_oracle import __all__  # noqa: F401
