"""FP64 CPU oracle for the PMACE hot path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; the product path never does.
"""
from . import pmace_oracle  # noqa: F401
