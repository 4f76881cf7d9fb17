"""CPU oracle (FP64, NumPy) for the consensus-ADMM calibration hot path.

TEST INFRASTRUCTURE. Importable only by the test suite, the package smoke check
and the benchmark's CPU-baseline / reference leg. The CUDA library never loads
it and shares no code with it.
"""
from . import admm

__all__ = ["admm"]
