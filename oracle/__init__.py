"""CPU FP64 oracle for the D3M dual block LDL^T factorization and solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA library and
never imports it; the product path does not call it.
"""
from .ldlt import *  # noqa: F401,F403
from .ldlt_bk import *  # noqa: F401,F403
