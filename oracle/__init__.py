"""FP64 CPU oracle for the NN-QST hot path (arXiv:2207.05341) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library and its Python binding never
do, and this package never imports them.
"""
from .qst_oracle import *  # noqa: F401,F403
from . import qst_oracle  # noqa: F401
