"""FP64 CPU oracle for non-linear digital tracking (arXiv 2503.08854, sec. 3).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the product path never does.  It shares
no code with the CUDA library (``paper_2503_08854_gb300``) and imports nothing
from it.  Parity of every function here is pinned by ``tests/test_oracle_*.py``.
"""
from .oracle import *  # noqa: F401,F403
