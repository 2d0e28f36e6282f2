"""Failure detection on the GPU: a bounded device wait that runs out is reported as an
error status and leaves the device usable.

The cooperative-grid Jacobi (revealed ranks whose r x r binary32 matrix exceeds one
CTA's shared memory) waits at a grid barrier after each rotating step.  The test lowers
the bound on that wait to one poll, so some CTA gives up at its first barrier; the
kernel then ends on every CTA with a status flag, and R4SVD must return SVT_ERR_CUDA
naming the grid Jacobi.  With the bound restored, the same call on the same device must
succeed and match the CPU oracle.  Nothing here faults, traps or hangs: the wait is
bounded by design and only the bound is changed.
"""
import numpy as np
import pytest

import oracle
from oracle import fastsvt as OF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt, torch


def test_grid_barrier_wait_runs_out_and_the_device_stays_usable(env):
    svt, torch = env
    from paper_1704_05528_gb300 import _lib as L
    lib = svt.library()
    rng = np.random.default_rng(41)
    m, n, z, r = 600, 500, 150_000, 200   # r = 200: 320 KB of binary32 A, above one CTA
    flat = rng.choice(m * n, size=z, replace=False)
    rows, cols = (flat // n).astype(np.int32), (flat % n).astype(np.int32)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    y = rng.standard_normal(ref_p.nnz)
    P = svt.Pattern(m, n, rows, cols)
    kw = dict(t=r, dt=10, n_power=0, r_max=r, seed=7)
    prev = lib.svt_test_set_grid_wait_limit(1)
    try:
        with pytest.raises(svt.SVTError) as e:
            svt.r4svd(P, torch.from_numpy(y), 1e-12, 1, **kw)
    finally:
        lib.svt_test_set_grid_wait_limit(prev)
    assert e.value.status == L.SVT_ERR_CUDA
    assert "grid Jacobi" in str(e.value)
    # the same device, the default bound: the call succeeds and matches the oracle
    got = svt.r4svd(P, torch.from_numpy(y), 1e-12, 1, **kw)
    ref = oracle.r4svd(OF._sparse(ref_p, y), None, 1e-12, 1, r_cap=r, t=r, dt=10, n_power=0, seed=7)
    assert got["r"] == ref.r == r
    S = got["S"].cpu().numpy()
    assert np.max(np.abs(S - ref.S)) / ref.S[0] < 1e-9
    torch.cuda.synchronize()

