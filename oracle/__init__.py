"""CPU oracle for microscopic avalanche transport (test infrastructure only).

Only tests/, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path (the CUDA library and its binding)
never does.
"""
from .oracle import *  # noqa: F401,F403
