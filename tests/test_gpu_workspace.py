"""Caller-owned workspaces: svt_complete, svt_complete_eval and svt_r4svd given a device
workspace of svt_workspace_size bytes allocate no device memory and return exactly what
the allocating calls return; a workspace that is too small is refused before any work.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt, torch


def _pool_high_water(torch):
    """Bytes in use in the device's default stream-ordered pool and its high-water mark
    (restarted), through the driver API; None where it cannot be read."""
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    pool = ctypes.c_void_p()
    if cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) != 0:
        return None
    cur = ctypes.c_uint64(0)
    if cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(cur)) != 0:  # USED_MEM_CURRENT
        return None
    if cu.cuMemPoolSetAttribute(pool, 8, ctypes.byref(ctypes.c_uint64(0))) != 0:  # restart USED_MEM_HIGH
        return None

    def high():
        h = ctypes.c_uint64(0)
        cu.cuMemPoolGetAttribute(pool, 8, ctypes.byref(h))
        return h.value
    return cur.value, high


def _same(a, b):
    to = lambda t: t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    assert a.iters == b.iters and a.k == b.k and a.r == b.r
    assert [e["r"] for e in a.log] == [e["r"] for e in b.log]
    assert [e["rel_residual"] for e in a.log] == [e["rel_residual"] for e in b.log]
    assert np.array_equal(to(a.U), to(b.U)) and np.array_equal(to(a.S), to(b.S))
    assert np.array_equal(to(a.V), to(b.V))


@pytest.mark.parametrize("prec,core_rows", [("fp64", 0), ("mixed", 0), ("mixed", 256)])
def test_complete_with_a_workspace_is_bit_identical_and_allocates_nothing(env, prec, core_rows):
    svt, torch = env
    w = workloads.ratings_6040(scale=0.3)
    kw = dict(t=w.t, dt=w.dt, beta=w.beta, eps_thr0=w.eps_thr0, r_max=w.r_max, seed=w.seed,
              n_power=w.n_power, core_rows=core_rows)
    vals = w.vals if prec == "fp64" else w.vals.astype(np.float32)
    d = lambda a: torch.from_numpy(a).cuda()
    ev = (w.held_rows, w.held_cols, w.held_vals if prec == "fp64" else w.held_vals.astype(np.float32))
    args = (w.m, w.n, d(w.rows), d(w.cols), d(vals), w.tau, w.delta, 0.0, 12)
    ref = svt.complete(*args, precision=prec, eval_set=ev, **kw)
    need = svt.workspace_size(w.m, w.n, w.nnz, n_eval=w.held_rows.size, precision=prec, **kw)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    svt.complete(*args, precision=prec, eval_set=ev, workspace=ws, **kw)  # first use
    torch.cuda.synchronize()
    pool = _pool_high_water(torch)
    free0 = torch.cuda.mem_get_info()[0]
    got = svt.complete(*args, precision=prec, eval_set=ev, workspace=ws, **kw)
    torch.cuda.synchronize()
    _same(got, ref)
    assert [e["mae_eval"] for e in got.log] == [e["mae_eval"] for e in ref.log]
    assert torch.cuda.mem_get_info()[0] == free0
    if pool is not None:
        cur0, high = pool
        assert high() == cur0


def test_complete_refuses_a_short_workspace_before_any_work(env):
    svt, torch = env
    w = workloads.random_lowrank(300, 200, 4, 0.3, seed=4, maxit=5)
    need = svt.workspace_size(w.m, w.n, w.nnz, t=10)
    ws = torch.full((need - 256,), 7, dtype=torch.uint8, device="cuda")
    with pytest.raises(svt.SVTError) as e:
        svt.complete(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, 0.0, 5, t=10, workspace=ws)
    from paper_1704_05528_gb300 import _lib as L
    assert e.value.status == L.SVT_ERR_ARG and "workspace" in str(e.value)
    assert bool((ws == 7).all())  # nothing was written into it


def test_r4svd_with_a_workspace(env):
    svt, torch = env
    w = workloads.small_lowrank()
    P = svt.Pattern(w.m, w.n, w.rows, w.cols)
    y = torch.from_numpy(np.random.default_rng(3).standard_normal(P.nnz)).cuda()
    kw = dict(t=25, dt=10, seed=w.seed)
    ref = svt.r4svd(P, y, 0.5, 1, **kw)
    ws = torch.empty(svt.r4svd_workspace_size(w.m, w.n, P.nnz, **kw), dtype=torch.uint8, device="cuda")
    got = svt.r4svd(P, y, 0.5, 1, workspace=ws, **kw)
    assert (got["r"], got["blocks"]) == (ref["r"], ref["blocks"])
    assert torch.equal(got["S"], ref["S"]) and torch.equal(got["U"], ref["U"])
    with pytest.raises(svt.SVTError):
        svt.r4svd(P, y, 0.5, 1, workspace=ws[:1024], **kw)
