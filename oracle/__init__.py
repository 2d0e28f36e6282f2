"""CPU oracle for fast SVT with R4SVD (plain numpy/scipy, FP64).

TEST INFRASTRUCTURE.  This package is the slow, obviously-correct restatement of
the method that the CUDA path is checked against.  Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline / reference legs of ``bench.py``
may import it; the product path never calls it and shares no code with it.
"""
from .philox import philox4x32_10, gaussian_block, PHILOX_M0, PHILOX_M1  # noqa: F401
from .fastsvt import (  # noqa: F401
    OracleError,
    Pattern,
    build_pattern,
    spectral_norm_estimate,
    householder_qr,
    r4svd,
    svt,
    d_tau_dense,
    sampled_product,
    SVTResult,
    R4SVDResult,
)
from .adjoint import (  # noqa: F401
    d_tau_jvp_dense,
    d_tau_dtau_dense,
    svt_unrolled_grad,
    UnrolledResult,
)
