"""svt_spmm_noalloc against svt_spmm.

The no-allocation variant exists for callers that cannot allocate device memory when
they need the product (another runtime has reserved the GPU's memory, or an allocation
would stall a latency-critical loop).  It must give the result of the ordinary entry
point, call after call, even though every call reuses the same fixed scratch array.
This file is collected last; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt, torch


def _pattern(svt, rng, m, n, z):
    flat = rng.choice(m * n, size=z, replace=False)
    rows, cols = (flat // n).astype(np.int32), (flat % n).astype(np.int32)
    return svt.Pattern(m, n, rows, cols)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_noalloc_matches_spmm_on_consecutive_calls(env, prec, tol):
    svt, torch = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(7)
    # two different problems back to back: the second call finds the first one's data in
    # the shared scratch array and must not be affected by it
    cases = [(_pattern(svt, rng, 611, 389, 30000), 100), (_pattern(svt, rng, 257, 1301, 20000), 10)]
    for P, width in cases:
        y = torch.from_numpy(rng.standard_normal(P.nnz)).to(device="cuda", dtype=dt)
        for transpose in (False, True):
            rows_in, rows_out = (P.m, P.n) if transpose else (P.n, P.m)
            W = torch.from_numpy(rng.standard_normal((rows_in, width))).to(device="cuda", dtype=dt)
            ref = svt.spmm(P, y, W, transpose=transpose, precision=prec)
            for _ in range(2):
                out = torch.full((rows_out, width), float("nan"), device="cuda", dtype=dt)
                svt.spmm_noalloc(P, y, W, out, transpose=transpose, precision=prec)
                err = (out - ref).norm().item() / max(ref.norm().item(), 1e-300)
                assert err <= tol


def test_noalloc_rejects_products_beyond_the_fixed_array(env):
    svt, torch = env
    from paper_1704_05528_gb300 import _lib as L
    rng = np.random.default_rng(8)
    P = _pattern(svt, rng, 2000, 1500, 400_000)
    y = torch.ones(P.nnz, device="cuda", dtype=torch.float64)
    W = torch.ones((P.m, 600), device="cuda", dtype=torch.float64)
    out = torch.zeros((P.n, 600), device="cuda", dtype=torch.float64)
    with pytest.raises(svt.SVTError) as e:
        svt.spmm_noalloc(P, y, W, out, transpose=True)
    assert e.value.status == L.SVT_ERR_UNSUPPORTED
    assert b"fixed array" in svt.library().svt_last_error()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_noalloc_takes_column_slices_of_wider_arrays(env, prec, tol):
    """W and out may be the first w columns of wider row-major arrays: the binding passes
    their row strides as leading dimensions, and the columns beyond w stay untouched."""
    svt, torch = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(9)
    P = _pattern(svt, rng, 523, 347, 25000)
    y = torch.from_numpy(rng.standard_normal(P.nnz)).to(device="cuda", dtype=dt)
    for width, ld in ((10, 12), (7, 16), (3, 3)):
        for transpose in (False, True):
            rows_in, rows_out = (P.m, P.n) if transpose else (P.n, P.m)
            Wb = torch.from_numpy(rng.standard_normal((rows_in, ld))).to(device="cuda", dtype=dt)
            ref = svt.spmm(P, y, Wb[:, :width].contiguous(), transpose=transpose, precision=prec)
            ob = torch.full((rows_out, ld + 2), float("nan"), device="cuda", dtype=dt)
            svt.spmm_noalloc(P, y, Wb[:, :width], ob[:, :width], transpose=transpose, precision=prec)
            err = (ob[:, :width] - ref).norm().item() / max(ref.norm().item(), 1e-300)
            assert err <= tol
            assert torch.isnan(ob[:, width:]).all()


def _default_pool_used(torch):
    """(current, high-water) bytes in use in the device's default stream-ordered pool,
    read through the driver API; None where the driver library cannot be loaded."""
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    pool = ctypes.c_void_p()
    if cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) != 0:
        return None
    used_current, used_high = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH
    cur, high = ctypes.c_uint64(0), ctypes.c_uint64(0)
    if cu.cuMemPoolGetAttribute(pool, used_current, ctypes.byref(cur)) != 0:
        return None
    if cu.cuMemPoolGetAttribute(pool, used_high, ctypes.byref(high)) != 0:
        return None
    return cu, pool, cur.value, high.value


def test_noalloc_allocates_no_device_memory(env):
    """The point of the entry point: repeated calls leave torch's allocator, the device's
    free memory and the default stream-ordered pool (whose high-water mark would catch an
    allocation freed before the call returns) exactly where they were."""
    svt, torch = env
    rng = np.random.default_rng(10)
    P = _pattern(svt, rng, 700, 450, 40000)
    y = torch.from_numpy(rng.standard_normal(P.nnz)).to(device="cuda", dtype=torch.float32)
    Wn = torch.from_numpy(rng.standard_normal((P.n, 12))).to(device="cuda", dtype=torch.float32)
    Wm = torch.from_numpy(rng.standard_normal((P.m, 12))).to(device="cuda", dtype=torch.float32)
    on = torch.empty((P.m, 12), device="cuda", dtype=torch.float32)
    ot = torch.empty((P.n, 12), device="cuda", dtype=torch.float32)
    # first calls: address lookup, and the kernels' code loaded on first launch
    svt.spmm_noalloc(P, y, Wn, on, precision="mixed")
    svt.spmm_noalloc(P, y, Wm, ot, transpose=True, precision="mixed")
    torch.cuda.synchronize()
    pool = _default_pool_used(torch)
    if pool is not None:
        cu, handle, cur0, _ = pool
        # restart the pool's high-water mark from the bytes in use now
        assert cu.cuMemPoolSetAttribute(handle, 8, ctypes.byref(ctypes.c_uint64(0))) == 0
    torch_before = torch.cuda.memory_allocated()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        svt.spmm_noalloc(P, y, Wn, on, precision="mixed")
        svt.spmm_noalloc(P, y, Wm, ot, transpose=True, precision="mixed")
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_before
    assert torch.cuda.mem_get_info()[0] == free_before
    if pool is not None:
        _, _, cur1, high1 = _default_pool_used(torch)
        assert cur1 == cur0 and high1 == cur0


def test_noalloc_rejects_short_operands_on_the_host(env):
    """The C entry point cannot see buffer sizes, so the binding refuses a W with the
    wrong number of rows or a y of the wrong length before anything is queued."""
    svt, torch = env
    rng = np.random.default_rng(11)
    P = _pattern(svt, rng, 300, 200, 5000)
    y = torch.zeros(P.nnz, device="cuda", dtype=torch.float64)
    out = torch.zeros((P.m, 4), device="cuda", dtype=torch.float64)
    with pytest.raises(ValueError):
        svt.spmm_noalloc(P, y, torch.zeros((P.n - 1, 4), device="cuda", dtype=torch.float64), out)
    with pytest.raises(ValueError):
        svt.spmm_noalloc(P, y[:-1], torch.zeros((P.n, 4), device="cuda", dtype=torch.float64), out)
    with pytest.raises(ValueError):
        svt.spmm(P, y, torch.zeros((P.n, 4), device="cuda", dtype=torch.float64), transpose=True)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_noalloc_matches_the_oracle_product(env, prec, tol):
    """The product of Algorithms 2-3 (X = Y Omega, and Y^T Q in the other order) against
    the binary64 oracle's sparse product on the same pattern and values, with a column
    spanning many work chunks (a popular column) so that the fix-up's segments run."""
    import oracle
    from oracle import fastsvt as OF
    svt, torch = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(23)
    m, n, z = 3000, 700, 60000
    flat = rng.choice(m * n, size=z, replace=False)
    rows, cols = (flat // n).astype(np.int32), (flat % n).astype(np.int32)
    extra = np.setdiff1d(np.arange(m, dtype=np.int64) * n + 5, flat)  # column 5 fully observed
    rows = np.concatenate([rows, (extra // n).astype(np.int32)])
    cols = np.concatenate([cols, (extra % n).astype(np.int32)])
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    y = rng.standard_normal(P.nnz)
    Ys = OF._sparse(ref_p, y)
    y_dev = torch.from_numpy(y).to(device="cuda", dtype=dt)
    for transpose, width in ((False, 10), (True, 100)):
        rows_in, rows_out = (m, n) if transpose else (n, m)
        W = rng.standard_normal((rows_in, width))
        W_dev = torch.from_numpy(W).to(device="cuda", dtype=dt)
        exact = np.asarray((Ys.T @ W) if transpose else (Ys @ W))
        for _ in range(2):
            out = torch.full((rows_out, width), float("nan"), device="cuda", dtype=dt)
            svt.spmm_noalloc(P, y_dev, W_dev, out, transpose=transpose, precision=prec)
            got = out.double().cpu().numpy()
            assert np.linalg.norm(got - exact) / np.linalg.norm(exact) <= tol
