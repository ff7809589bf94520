"""FP64 CPU oracle for PRGD tensor-train completion.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: it is used by `tests/`, by `__graft_entry__.smoke()` (to check one
GPU step) and by the CPU-baseline leg of `bench.py`.  It shares no code with
the CUDA library.
"""
from .prgd import *  # noqa: F401,F403
