"""CPU oracle for the ensemble channel DNS step -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of the paper's method (operators built in
IEEE quad precision, rounded once to double).  Only the tests, the smoke check
and the benchmark's CPU-baseline / reference leg may import it.  It shares no
code with the GPU library and never calls it.
"""
from .dns import (Channel, RK3_SUBSTEPS, cn_rk3, grid, cc_weights, cn_operators,  # noqa: F401
                  mean_operators, quad_solve, fundamental)
from .linear import Linear  # noqa: F401
