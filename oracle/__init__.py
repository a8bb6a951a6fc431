"""CPU oracle (FP64) for the nodal H-field FE method.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import it.  The library itself never
imports, links or runs anything here, and the two share no code.
"""
from . import fem, krylov, precond  # noqa: F401
