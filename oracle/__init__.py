"""FP64 CPU oracle of the KFAC-for-PINNs hot path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this package; the library never does.
"""
from . import kfac_oracle  # noqa: F401
