"""svt_spmm_noalloc against svt_spmm.

The no-allocation variant exists for callers that cannot allocate device memory when
they need the product (another runtime has reserved the GPU's memory, or an allocation
would stall a latency-critical loop).  It must give the result of the ordinary entry
point, call after call, even though every call reuses the same fixed scratch array.
This file is collected last; it also passes on its own in a fresh process.
"""
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
