"""FP64 CPU oracle for the randomized Tucker path (arXiv 2303.11612).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg are the only code that may import this package. The CUDA
library never imports, links or calls it, and it never calls the library.

Every function here is pinned by a ``-m "not gpu"`` test to something other
than itself (published Philox answers, brute-force sums, closed forms, bounds
stated in the paper, library routines on special cases, exhaustive enumeration
of sampling outcomes). Pinned parts: see tests/test_oracle_*.py.
"""
from . import philox, tucker  # noqa: F401
