"""Seeded synthetic matrix-completion inputs.

This package only draws inputs: index sets, observed values, held-out entries and
the solver parameters that go with each workload.  It holds none of the method's
arithmetic (no SVD, no thresholding, no sparse products), so the CPU oracle and the
CUDA path can both be fed from it without sharing any of the computation.

The five workloads stand in for the paper's data sets, which are not available:
a small rank-10 problem, a 512x512 image-like problem (Section 3.1 uses a
512x512 grayscale image), two rating matrices shaped like MovieLens (Section 3.2)
and a 2000x2000 problem for the unrolled, differentiated solver.
"""
from .synth import (  # noqa: F401
    Workload,
    WORKLOADS,
    make,
    small_lowrank,
    image_512,
    ratings_6040,
    ratings_71567,
    ratings,
    unrolled_2000,
    random_lowrank,
)
