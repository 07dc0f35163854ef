"""FP64 CPU oracle of the moving-boundary lattice electrokinetics step.

Test infrastructure only: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the product path never does.
"""
from .ek_oracle import EKOracle, OracleError  # noqa: F401
