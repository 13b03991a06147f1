"""GB300 Schur-complement solver for block-arrowhead KKT systems.

The C ABI (include/kkt_schur.h) is implemented by the CUDA library built from
csrc/ (paper_1907_05420_gb300/_build/libkkt_schur.so); `binding` is a thin
ctypes layer over it with the same function names.
"""
from .binding import (  # noqa: F401
    KKT_BF16,
    KKT_F64_EMULATED,
    KKT_FP64,
    KKT_TF32,
    KKTError,
    KKTSolver,
    kkt_analyze,
    kkt_default_options,
    kkt_destroy,
    kkt_factor,
    kkt_get_info,
    kkt_solve,
    load,
)
