"""FP64 CPU oracle of the Bloch-wave hot path.

Test infrastructure: only tests/, the package smoke check and the CPU-baseline
leg of bench.py may import this package.  It shares no code with the CUDA path.
"""
from . import bloch_oracle, closed_forms  # noqa: F401
