"""FP64 CPU oracle of the relativistic lattice Boltzmann update.

Test infrastructure only: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product path.
"""
from .rlbm_oracle import *  # noqa: F401,F403
