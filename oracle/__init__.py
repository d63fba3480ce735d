"""FP64 CPU oracle of the (DD) parabolic Monge-Ampere mesh generator.

TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke test and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  It wraps the plain C implementation in ``pma_oracle.c`` (built with
``build()``) and shares no code with the CUDA library: problem descriptions
are read by attribute from the seeded input module, nothing else is shared.
"""
from .oracle import (build, lib_path, solve, solve_parallel, operator, monitor_eval,
                     extents, quality, OracleResult)

__all__ = ["build", "lib_path", "solve", "solve_parallel", "operator", "monitor_eval", "extents",
           "quality", "OracleResult"]
