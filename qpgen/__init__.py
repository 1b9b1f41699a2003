"""Seeded synthetic QP workloads.

This package only draws random problem data (numpy, FP64, rounded to FP32 on
request).  It holds none of the solver's arithmetic, so both the FP64 oracle
tests and the CUDA path can take their inputs from it.
"""
from .workloads import (  # noqa: F401
    CONFIGS,
    QPBatch,
    instance_rng,
    make_batch,
    make_instance,
    serving_sizes,
)
