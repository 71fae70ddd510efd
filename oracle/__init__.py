"""CPU oracle (FP64 / int64) -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library and never calls it.
"""
from .oracle import *  # noqa: F401,F403
