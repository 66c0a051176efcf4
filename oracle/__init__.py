"""FP64 CPU oracle for extended RaBitQ (arXiv 2409.09913).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg are the only permitted users.  Nothing here is imported by,
or imports, the GPU package.
"""
from .oracle import *  # noqa: F401,F403
