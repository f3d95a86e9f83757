"""FP64 CPU oracle of the DLMPC ADMM (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline/reference
arm import this package; the library never does.
"""
from .dlmpc_oracle import *  # noqa: F401,F403
