"""FP64 CPU oracle for kernel quantile regression (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it.
"""
from .kqr_oracle import *  # noqa: F401,F403
