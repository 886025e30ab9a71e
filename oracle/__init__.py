"""Plain FP64 CPU oracle for the constrained-realization fill-in.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may use it.  It shares no code with the CUDA path.
"""
from .cgfill_oracle import *  # noqa: F401,F403
