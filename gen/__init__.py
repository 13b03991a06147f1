"""Seeded synthetic inputs for the block-arrowhead KKT solve.

This package only builds inputs: grids, the per-period blocks A_i, the
coupling blocks B_i, the coupling diagonal C and right-hand sides.  It holds
none of the Schur-complement method's arithmetic, so both the CUDA path and
the CPU oracle can draw their inputs from it without sharing method code.
"""
from .mpopf import (  # noqa: F401
    GridSpec,
    KKTProblem,
    CONFIGS,
    make_problem,
    mix_spec,
    reseed_barrier,
)
from .scopf import make_scopf  # noqa: F401
from .ipm import make_ipm_state  # noqa: F401
from .workloads import build_workload, describe_workload, is_workload  # noqa: F401
