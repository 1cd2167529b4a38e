"""FP64 CPU oracle for the quantization-based Wasserstein bounds.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the library.
"""
from .qwb_oracle import *  # noqa: F401,F403
from . import qwb_oracle  # noqa: F401
