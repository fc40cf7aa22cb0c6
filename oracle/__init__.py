"""FP64 CPU oracle of piCholesky cross-validation.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline of the benchmark, never by the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, cv, CVResult, NotSPD  # noqa: F401
