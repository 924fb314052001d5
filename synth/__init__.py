"""Seeded synthetic inputs for DPar2 workloads.

This package only *generates inputs*: irregular dense tensors shaped like the
paper's workloads, Gaussian test matrices and initial factors.  It holds none
of the decomposition's arithmetic, and both the CUDA path's tests/benchmark
and the FP64 oracle draw their inputs from here.
"""
from .generators import (  # noqa: F401
    WORKLOADS,
    Workload,
    bf16_representable,
    gaussian_matrix,
    make_row_offsets,
    plain_parafac2,
    spectrogram_like,
    stock_factors,
    skewed_series,
    tenrand,
    workload,
)
