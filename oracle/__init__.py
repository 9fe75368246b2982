"""Dense FP64 CPU oracle (test infrastructure only).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may
import this package; the library never does.  See gnk_dense for what it
computes and which parts of the paper each function follows.
"""
from . import gnk_dense  # noqa: F401
