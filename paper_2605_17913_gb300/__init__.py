"""Batched, differentiable FP32 interior-point QP solver with implicit
complementarity for NVIDIA GB300 (sm_103a).

Method: "A Differentiable Interior-Point Method in Single Precision"
(Alg. 1 solve, Alg. 2 relax, Alg. 3 gradients).  The C ABI is in
include/qp.h; this package is a thin binding over it.
"""
from ._lib import (  # noqa: F401
    QP_BAD_INPUT, QP_MAX_ITER, QP_NUMERICAL, QP_SOLVED, QP_STALLED, QPError, default_settings,
    lib, smem_bytes, status_string,
)


def __getattr__(name):
    # torch-dependent parts load lazily so that the binding can be inspected without a GPU
    if name in ("QPSolver", "QPFunction", "qp_layer", "get_solver"):
        from . import solver

        return getattr(solver, name)
    raise AttributeError(name)
