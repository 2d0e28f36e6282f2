"""CUDA path (through the C ABI) against the CPU oracle on identical seeded inputs.

Bars: bit-exact for the pattern (integer work) and for the per-iteration revealed
rank / kept count in binary64; relative 1e-9 for singular values and completed
entries in binary64; relative Frobenius 1e-3 in mixed precision.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import fastsvt as OF

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-3


@pytest.fixture(scope="module")
def svt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))


def _coo(rng, m, n, z):
    flat = rng.choice(m * n, size=z, replace=False)
    return (flat // n).astype(np.int32), (flat % n).astype(np.int32)


# --------------------------------------------------------------------- pattern
PATTERN_KEYS = ("row_ptr", "col_idx", "csr_src", "col_ptr", "row_idx", "perm")


def _check_pattern(svt, m, n, rows, cols):
    P = svt.Pattern(m, n, rows, cols)
    got = {k: v.cpu().numpy() for k, v in P.export().items()}
    ref = oracle.build_pattern(m, n, rows, cols)
    for k in PATTERN_KEYS:
        assert np.array_equal(got[k], getattr(ref, k)), k


@pytest.mark.parametrize("m,n,z", [(7, 5, 12), (1, 9, 4), (9, 1, 5), (13, 17, 0), (1, 1, 1),
                                   (300, 200, 5000), (2049, 3, 6000), (3, 5000, 14000)])
def test_pattern_bit_exact(svt, m, n, z):
    rng = np.random.default_rng(m * 7 + n)
    rows, cols = _coo(rng, m, n, z)
    _check_pattern(svt, m, n, rows, cols)


def test_pattern_dense_rows_and_empty_rows(svt):
    m, n = 40, 3000
    rows = np.concatenate([np.full(n, 5), np.full(n, 33), np.arange(0, 40, 7)]).astype(np.int32)
    cols = np.concatenate([np.arange(n), np.arange(n)[::-1], np.arange(0, 40, 7) + 1]).astype(np.int32)
    _check_pattern(svt, m, n, rows, cols)


def test_pattern_errors(svt):
    from paper_1704_05528_gb300 import _lib as L
    for rows, cols, want in [([0, 1, 1], [0, 2, 2], L.SVT_ERR_DUPLICATE),
                             ([0, 4], [0, 1], L.SVT_ERR_INDEX),
                             ([0, 1], [0, -1], L.SVT_ERR_INDEX)]:
        with pytest.raises(svt.SVTError) as e:
            svt.Pattern(4, 4, np.array(rows, np.int32), np.array(cols, np.int32))
        assert e.value.status == want


# ------------------------------------------------------------------ Gaussians
@pytest.mark.parametrize("n,w", [(1, 1), (10, 1), (1000, 10), (777, 7), (5, 64)])
def test_gaussian_block(svt, n, w):
    got = svt.gaussian_block(0x5EED, 3, 2, n, w).cpu().numpy()
    ref = oracle.gaussian_block(0x5EED, 3, 2, n, w)
    # same Philox words; Box-Muller through CUDA's and libm's log/sqrt/sin/cos
    assert np.max(np.abs(got - ref)) < 1e-13


# ------------------------------------------------------------------------ SpMM
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
@pytest.mark.parametrize("width", [1, 3, 10, 33, 100, 513, 600])
def test_spmm(svt, torch_mod, prec, tol, width):
    rng = np.random.default_rng(width)
    m, n = 611, 389
    rows, cols = _coo(rng, m, n, 30000)
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    y = rng.standard_normal(ref_p.nnz)
    dt = np.float64 if prec == "fp64" else np.float32
    y = y.astype(dt).astype(np.float64)
    Ys = OF._sparse(ref_p, y)
    W = rng.standard_normal((n, width)).astype(dt)
    W2 = rng.standard_normal((m, width)).astype(dt)
    got = svt.spmm(P, torch_mod.from_numpy(y.astype(dt)), torch_mod.from_numpy(W), precision=prec)
    got2 = svt.spmm(P, torch_mod.from_numpy(y.astype(dt)), torch_mod.from_numpy(W2), transpose=True,
                    precision=prec)
    assert _rel(got.cpu().numpy(), Ys @ W.astype(np.float64)) < tol
    assert _rel(got2.cpu().numpy(), Ys.T @ W2.astype(np.float64)) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
def test_spmm_narrow_widths_on_skewed_rows(svt, torch_mod, prec, tol):
    """Widths 1-16 take the entry-segmented kernel: rows of thousands of entries that span
    many chunks, empty rows and columns, and short rows, in both orders."""
    rng = np.random.default_rng(77)
    m, n = 900, 700
    heavy_r = np.repeat(np.array([3, 450, 899], np.int32), 600)
    heavy_c = np.concatenate([rng.choice(n, 600, replace=False) for _ in range(3)]).astype(np.int32)
    flat = rng.choice(m * n, size=20000, replace=False)
    rows = np.concatenate([heavy_r, (flat // n).astype(np.int32)])
    cols = np.concatenate([heavy_c, (flat % n).astype(np.int32)])
    keep = (rows % 7 != 5) & (cols % 11 != 4)            # some empty rows and columns
    key = rows.astype(np.int64) * n + cols
    _, first = np.unique(key, return_index=True)          # distinct entries only
    sel = np.zeros(rows.size, bool)
    sel[first] = True
    sel &= keep
    rows, cols = rows[sel], cols[sel]
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    dt = np.float64 if prec == "fp64" else np.float32
    y = rng.standard_normal(ref_p.nnz).astype(dt)
    Ys = OF._sparse(ref_p, y.astype(np.float64))
    for width in (1, 2, 3, 4, 5, 8, 10, 12, 16):
        W = rng.standard_normal((n, width)).astype(dt)
        W2 = rng.standard_normal((m, width)).astype(dt)
        got = svt.spmm(P, torch_mod.from_numpy(y), torch_mod.from_numpy(W), precision=prec)
        got2 = svt.spmm(P, torch_mod.from_numpy(y), torch_mod.from_numpy(W2), transpose=True, precision=prec)
        assert _rel(got.cpu().numpy(), Ys @ W.astype(np.float64)) < tol, width
        assert _rel(got2.cpu().numpy(), Ys.T @ W2.astype(np.float64)) < tol, width


# ---------------------------------------------------------- sampled update
@pytest.mark.parametrize("k", [0, 1, 10, 37])
def test_sampled_update(svt, torch_mod, k):
    rng = np.random.default_rng(100 + k)
    m, n = 301, 257
    rows, cols = _coo(rng, m, n, 9000)
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    U = rng.standard_normal((m, k))
    Wm = rng.standard_normal((n, k))
    a = rng.standard_normal(ref_p.nnz)
    y0 = rng.standard_normal(ref_p.nnz)
    delta = 1.7
    x = oracle.sampled_product(U, np.ones(k), Wm, ref_p.csr_rows(), ref_p.col_idx)
    d = a - x
    y_ref = y0 + delta * d
    y_dev = torch_mod.from_numpy(y0.copy()).cuda()
    sums = svt.sampled_update(P, torch_mod.from_numpy(U), torch_mod.from_numpy(Wm),
                              torch_mod.from_numpy(a), y_dev, delta)
    assert _rel(y_dev.cpu().numpy(), y_ref) < 1e-14
    assert math.isclose(sums[0], float(np.sum(d * d)), rel_tol=1e-12)
    assert math.isclose(sums[1], float(np.sum(np.abs(d))), rel_tol=1e-12)
    assert math.isclose(sums[2], float(np.sum(y_ref * y_ref)), rel_tol=1e-12)


@pytest.mark.parametrize("k", [4, 60, 100, 128, 132, 7])
def test_sampled_update_mixed(svt, torch_mod, k):
    """Binary32 update on a pattern with heavy columns (40 columns holding 24,000 entries),
    an empty column range and a narrow last block of columns; k = 7 has unaligned rows
    (scalar loads), the others take the float4 path."""
    rng = np.random.default_rng(7 + k)
    m, n = 3001, 1300
    heavy = rng.choice(m * 40, size=24000, replace=False)
    other_cols = np.setdiff1d(np.arange(40, n), np.arange(512, 768))
    flat_o = rng.choice(m * other_cols.size, size=36000, replace=False)
    rows = np.concatenate([heavy // 40, flat_o // other_cols.size]).astype(np.int32)
    cols = np.concatenate([heavy % 40, other_cols[flat_o % other_cols.size]]).astype(np.int32)
    perm = rng.permutation(rows.size)
    rows, cols = rows[perm], cols[perm]
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    f32 = lambda x: np.asarray(x, dtype=np.float32)
    U = f32(rng.standard_normal((m, k)))
    Wm = f32(rng.standard_normal((n, k)))
    a = f32(rng.standard_normal(ref_p.nnz))
    y0 = f32(rng.standard_normal(ref_p.nnz))
    delta = 1.7
    x = oracle.sampled_product(U.astype(np.float64), np.ones(k), Wm.astype(np.float64),
                               ref_p.csr_rows(), ref_p.col_idx)
    d = a.astype(np.float64) - x
    y_ref = y0.astype(np.float64) + delta * d
    y_dev = torch_mod.from_numpy(y0.copy()).cuda()
    sums = svt.sampled_update(P, torch_mod.from_numpy(U), torch_mod.from_numpy(Wm),
                              torch_mod.from_numpy(a), y_dev, delta, precision="mixed")
    got = y_dev.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - y_ref)) < 1e-5 * (1.0 + np.sqrt(k)) * delta
    assert math.isclose(sums[0], float(np.sum(d * d)), rel_tol=1e-5)
    assert math.isclose(sums[1], float(np.sum(np.abs(d))), rel_tol=1e-5)
    assert math.isclose(sums[2], float(np.sum(y_ref * y_ref)), rel_tol=1e-5)


def _recycle_case(rng, m, n):
    """Heavy columns (40 columns holding 24,000 entries, each spanning many entry chunks),
    an empty column range inside and at the end, scattered entries elsewhere."""
    heavy = rng.choice(m * 40, size=24000, replace=False)
    other_cols = np.setdiff1d(np.arange(40, n - 5), np.arange(512, 768))
    flat_o = rng.choice(m * other_cols.size, size=36000, replace=False)
    rows = np.concatenate([heavy // 40, flat_o // other_cols.size]).astype(np.int32)
    cols = np.concatenate([heavy % 40, other_cols[flat_o % other_cols.size]]).astype(np.int32)
    perm = rng.permutation(rows.size)
    return rows[perm], cols[perm]


def _recycle_reference(ref_p, n, U, Wm, a, y0, delta):
    """Y_new in CSC order (eq. (5) on Lambda) and B^T = Y_new^T U, in binary64."""
    import scipy.sparse as sp
    k = Wm.shape[1]
    cols = np.repeat(np.arange(n), np.diff(ref_p.col_ptr))
    x = oracle.sampled_product(U[:, :k], np.ones(k), Wm, ref_p.row_idx, cols)
    d = a - x
    y_new = y0 + delta * d
    Yt = sp.csr_matrix((y_new, (cols, ref_p.row_idx)), shape=(n, U.shape[0]))
    bound = sp.csr_matrix((np.abs(y_new), (cols, ref_p.row_idx)), shape=(n, U.shape[0])) @ np.abs(U)
    return y_new, d, Yt @ U, bound


@pytest.mark.parametrize("r,k", [(100, 60), (8, 8), (130, 0), (256, 200), (1, 1)])
def test_sampled_update_recycle(svt, torch_mod, r, k):
    """The fused CSC-order update and recycled product against the binary64 definitions."""
    rng = np.random.default_rng(31 + r + k)
    m, n = 3001, 1300
    rows, cols = _recycle_case(rng, m, n)
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    U = rng.standard_normal((m, r))
    Wm = rng.standard_normal((n, k))
    a = rng.standard_normal(ref_p.nnz)
    y0 = rng.standard_normal(ref_p.nnz)
    delta = 1.3
    y_ref, d, bt_ref, bound = _recycle_reference(ref_p, n, U, Wm, a, y0, delta)
    y_dev = torch_mod.from_numpy(y0.copy()).cuda()
    Bt, sums = svt.sampled_update_recycle(P, torch_mod.from_numpy(U), torch_mod.from_numpy(Wm),
                                          torch_mod.from_numpy(a), y_dev, delta)
    assert _rel(y_dev.cpu().numpy(), y_ref) < 1e-14
    assert np.all(np.abs(Bt.cpu().numpy() - bt_ref) <= 1e-13 * bound + 1e-300)
    assert not np.any(Bt.cpu().numpy()[512:768]) and not np.any(Bt.cpu().numpy()[n - 5:])
    assert math.isclose(sums[0], float(np.sum(d * d)), rel_tol=1e-12)
    assert math.isclose(sums[1], float(np.sum(np.abs(d))), rel_tol=1e-12)
    assert math.isclose(sums[2], float(np.sum(y_ref * y_ref)), rel_tol=1e-12)


@pytest.mark.parametrize("r,k", [(100, 60), (100, 100), (3, 2), (64, 33), (200, 128), (512, 300),
                                 (130, 0)])
def test_sampled_update_recycle_mixed(svt, torch_mod, r, k):
    rng = np.random.default_rng(57 + r + k)
    m, n = 3001, 1300
    rows, cols = _recycle_case(rng, m, n)
    P = svt.Pattern(m, n, rows, cols)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    f32 = lambda x: np.asarray(x, dtype=np.float32)
    U = f32(rng.standard_normal((m, r)) / np.sqrt(r))
    Wm = f32(rng.standard_normal((n, k)))
    a = f32(rng.standard_normal(ref_p.nnz))
    y0 = f32(rng.standard_normal(ref_p.nnz))
    delta = 1.3
    y_ref, d, bt_ref, bound = _recycle_reference(ref_p, n, U.astype(np.float64), Wm.astype(np.float64),
                                                 a.astype(np.float64), y0.astype(np.float64), delta)
    y_dev = torch_mod.from_numpy(y0.copy()).cuda()
    Bt, sums = svt.sampled_update_recycle(P, torch_mod.from_numpy(U), torch_mod.from_numpy(Wm),
                                          torch_mod.from_numpy(a), y_dev, delta, precision="mixed")
    got = y_dev.cpu().numpy().astype(np.float64)
    # binary32 dot of k terms: error below k ulps of sum |u w|, here (1 + sqrt(k)) delta 1e-5
    assert np.max(np.abs(got - y_ref)) < 1e-5 * (1.0 + np.sqrt(k)) * delta
    # each B^T element: binary32 sum over its column of y_new U, with y_new itself rounded
    err = np.abs(Bt.cpu().numpy().astype(np.float64) - bt_ref)
    assert np.all(err <= 1e-5 * (1.0 + np.sqrt(k)) * bound + 1e-30)
    assert math.isclose(sums[0], float(np.sum(d * d)), rel_tol=1e-5)
    assert math.isclose(sums[1], float(np.sum(np.abs(d))), rel_tol=1e-5)
    assert math.isclose(sums[2], float(np.sum(y_ref * y_ref)), rel_tol=1e-5)


# ------------------------------------------------------------------------ R4SVD
def _sigma_close(got, ref, tol):
    got = np.asarray(got)
    assert got.shape == ref.shape
    return float(np.max(np.abs(got - ref)) / ref[0]) < tol


@pytest.mark.parametrize("eps_thr,n_power", [(0.9, 0), (0.5, 0), (0.6, 1)])
def test_r4svd_parity(svt, torch_mod, eps_thr, n_power):
    w = workloads.small_lowrank()
    ref_p = oracle.build_pattern(w.m, w.n, w.rows, w.cols)
    P = svt.Pattern(w.m, w.n, w.rows, w.cols)
    y = w.vals[ref_p.csr_src] * 12.0
    Ys = OF._sparse(ref_p, y)
    kw = dict(t=25, dt=10, n_power=n_power)
    ro = oracle.r4svd(Ys, None, eps_thr, 1, r_cap=500, seed=w.seed, **kw)
    rg = svt.r4svd(P, torch_mod.from_numpy(y), eps_thr, 1, seed=w.seed, **kw)
    assert (rg["r"], rg["blocks"]) == (ro.r, ro.blocks)
    assert abs(rg["eps"] - ro.eps) < 1e-12
    assert _sigma_close(rg["S"].cpu().numpy(), ro.S, FP64_TOL)
    # recycled call (Algorithm 3) from each side's own basis
    ro2 = oracle.r4svd(Ys, ro.U, eps_thr * 0.5, 2, r_cap=500, seed=w.seed, **kw)
    rg2 = svt.r4svd(P, torch_mod.from_numpy(y), eps_thr * 0.5, 2, U_prev=rg["U"], seed=w.seed, **kw)
    assert (rg2["r"], rg2["blocks"]) == (ro2.r, ro2.blocks)
    S2 = rg2["S"].cpu().numpy()
    assert _sigma_close(S2, ro2.S, FP64_TOL)
    k = 10  # the rank-10 part is well separated: compare the reconstruction
    Xo = (ro2.U[:, :k] * ro2.S[:k]) @ ro2.V[:, :k].T
    Xg = (rg2["U"][:, :k].cpu().numpy() * S2[:k]) @ rg2["V"][:, :k].cpu().numpy().T
    assert _rel(Xg, Xo) < FP64_TOL


@pytest.mark.parametrize("r_max", [100, 128, 16, 40, 150])
def test_r4svd_mixed_lift(svt, torch_mod, r_max):
    """Binary32 R4SVD: U = Q U_B runs on the tensor cores (three TF32 products per term)
    for r <= 128 and on the binary32 SIMT kernel above that.  1,000 rows span eight
    128-row tiles and a ragged tail; the basis must stay orthonormal and the well-separated
    rank-10 part must match the binary64 oracle."""
    w = workloads.random_lowrank(1000, 300, 10, 0.3, seed=21)
    ref_p = oracle.build_pattern(w.m, w.n, w.rows, w.cols)
    P = svt.Pattern(w.m, w.n, w.rows, w.cols)
    y = w.vals[ref_p.csr_src] * 12.0
    Ys = OF._sparse(ref_p, y)
    kw = dict(t=min(r_max, 30), dt=10, n_power=0)
    ro = oracle.r4svd(Ys, None, 1e-12, 1, r_cap=r_max, seed=w.seed, **kw)
    rg = svt.r4svd(P, torch_mod.from_numpy(y), 1e-12, 1, seed=w.seed, r_max=r_max,
                   precision="mixed", **kw)
    assert rg["r"] == ro.r == r_max
    U = rg["U"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(U.T @ U - np.eye(r_max))) < 2e-5
    S = rg["S"].cpu().numpy()
    k = 10
    assert np.max(np.abs(S[:k] - ro.S[:k])) / ro.S[0] < 1e-5
    Xo = (ro.U[:, :k] * ro.S[:k]) @ ro.V[:, :k].T
    Xg = (U[:, :k] * S[:k]) @ rg["V"][:, :k].cpu().numpy().astype(np.float64).T
    assert _rel(Xg, Xo) < 1e-4


def _oracle_state(w, it_stop, **kw):
    """(Y in CSR order at SVT iteration it_stop, the basis that iteration recycles), from
    the oracle's own solve."""
    captured = {}
    orig = OF.r4svd

    def spy(Ys, U_prev, eps_thr, it, **kws):
        if it == it_stop:
            captured["y"] = Ys
            captured["U_prev"] = None if U_prev is None else np.array(U_prev)
            captured["eps_thr"] = eps_thr
        return orig(Ys, U_prev, eps_thr, it, **kws)
    OF.r4svd = spy
    try:
        OF.svt(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, 0.0, it_stop, seed=w.seed, **kw)
    finally:
        OF.r4svd = orig
    return captured


@pytest.mark.parametrize("name,it_stop,kw", [
    ("recovery40", 206, dict(eps_thr0=1e-12)),
    ("recovery40", 8, dict(eps_thr0=1e-12)),
    ("lowrank500", 30, dict()),
])
def test_r4svd_recycled_near_diagonal(svt, torch_mod, name, it_stop, kw):
    """Recycled calls start the binary64 refinement from the near-diagonal Gram matrix
    (coupled clusters diagonalised); every singular value must still match the oracle.
    At iteration 8 of the 40 x 40 recovery, clusters of 23, 10 and 3 leave a coupled pair
    unresolved, and the result must come from the Jacobi fallback."""
    if name == "recovery40":
        w = workloads.random_lowrank(40, 40, 2, 0.6, seed=33, tol=1e-9, maxit=1000)
    else:
        w = workloads.small_lowrank()
    st = _oracle_state(w, it_stop, **kw)
    ref_p = oracle.build_pattern(w.m, w.n, w.rows, w.cols)
    Ys = st["y"].tocsr()
    y = np.asarray(Ys[ref_p.csr_rows(), ref_p.col_idx]).ravel()
    P = svt.Pattern(w.m, w.n, w.rows, w.cols)
    U_prev = st["U_prev"]
    ro = oracle.r4svd(Ys, U_prev, st["eps_thr"], it_stop, r_cap=min(w.m, w.n), seed=w.seed, t=1,
                      dt=10, n_power=0)
    rg = svt.r4svd(P, torch_mod.from_numpy(y), st["eps_thr"], it_stop, U_prev=torch_mod.from_numpy(U_prev),
                   seed=w.seed, dt=10)
    assert (rg["r"], rg["blocks"]) == (ro.r, ro.blocks)
    S = rg["S"].cpu().numpy()
    assert np.max(np.abs(S - ro.S)) / ro.S[0] < FP64_TOL, (S[:4], ro.S[:4])


def test_r4svd_exhausted_range(svt, torch_mod):
    """A rank-3 matrix with a full pattern and a threshold no error percentage can meet:
    the block after the first finds the range exhausted and is discarded."""
    rng = np.random.default_rng(5)
    m, n = 40, 30
    M = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n))
    rows, cols = np.nonzero(np.ones((m, n)))
    rows, cols = rows.astype(np.int32), cols.astype(np.int32)
    ref_p = oracle.build_pattern(m, n, rows, cols)
    y = M[ref_p.csr_rows(), ref_p.col_idx]
    ro = oracle.r4svd(OF._sparse(ref_p, y), None, -1.0, 1, t=3, dt=2, n_power=0, r_cap=30, seed=2)
    P = svt.Pattern(m, n, rows, cols)
    rg = svt.r4svd(P, torch_mod.from_numpy(y), -1.0, 1, t=3, dt=2, seed=2)
    assert ro.exhausted and ro.r == 3 and rg["r"] == 3 and rg["blocks"] == ro.blocks
    assert _sigma_close(rg["S"].cpu().numpy(), ro.S, FP64_TOL)


# ---------------------------------------------------------------- fast SVT
def _run_pair(svt, torch_mod, w, maxit, prec, tol=None, **over):
    kw = dict(t=w.t, dt=w.dt, beta=w.beta, eps_thr0=w.eps_thr0, r_max=w.r_max, seed=w.seed,
              n_power=w.n_power)
    kw.update(over)
    tol = w.tol if tol is None else tol
    ref = oracle.svt(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, tol, maxit, **kw)
    vals = w.vals if prec == "fp64" else w.vals.astype(np.float32)
    got = svt.complete(w.m, w.n, torch_mod.from_numpy(w.rows).cuda(), torch_mod.from_numpy(w.cols).cuda(),
                       torch_mod.from_numpy(vals).cuda(), w.tau, w.delta, tol, maxit, precision=prec, **kw)
    return ref, got


def _completed(res_U, res_S, res_V, rows, cols):
    to = lambda t: t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    return oracle.sampled_product(to(res_U), to(res_S), to(res_V), rows, cols)


def _assert_fp64_parity(w, ref, got):
    assert got.iters == ref.iters and got.k == ref.k and got.k0 == ref.k0
    assert [e["r"] for e in got.log] == [e["r"] for e in ref.log]
    assert [e["k"] for e in got.log] == [e["k"] for e in ref.log]
    assert [e["blocks"] for e in got.log] == [e["blocks"] for e in ref.log]
    assert [bool(e["cooled"]) for e in got.log] == [e["cooled"] for e in ref.log]
    p = ref.pattern
    x_obs_ref = _completed(ref.U, ref.S, ref.V, p.csr_rows(), p.col_idx)
    x_obs_got = _completed(got.U, got.S, got.V, p.csr_rows(), p.col_idx)
    assert _rel(x_obs_got, x_obs_ref) < FP64_TOL
    if w.held_rows.size:
        x_h_ref = _completed(ref.U, ref.S, ref.V, w.held_rows, w.held_cols)
        x_h_got = _completed(got.U, got.S, got.V, w.held_rows, w.held_cols)
        assert _rel(x_h_got, x_h_ref) < FP64_TOL
    s_got = got.S.cpu().numpy() if hasattr(got.S, "cpu") else got.S
    if ref.k:
        assert np.max(np.abs(s_got - ref.S) / (ref.S + w.tau)) < FP64_TOL


def test_complete_fp64_above_fused_rank(svt, torch_mod):
    """Revealed rank above the fused update's binary64 limit (256 columns): the solver
    switches to the CSR-order sampled update, keeps the CSC copy of Y by regathering it,
    and refreshes the CSR copy when the fused pass wrote only the CSC one."""
    w = workloads.random_lowrank(420, 380, 6, 0.5, seed=17, maxit=8, tol=1e-12)
    w.tau = np.sqrt(w.m * w.n)  # keeps the separated rank-6 part (k = 5-6)
    ref, got = _run_pair(svt, torch_mod, w, w.maxit, "fp64", t=240, dt=12, r_max=300,
                         eps_thr0=0.05)
    rs = [e["r"] for e in ref.log]
    assert min(rs) <= 256 < max(rs), rs  # both the fused and the CSR-order update ran
    _assert_fp64_parity(w, ref, got)


@pytest.mark.parametrize("recycle,over", [
    ("kept", {}),
    ("none", {}),
    ("none", {"t": 30, "r_max": 30, "n_power": 1}),   # fixed-rank randomized SVD
])
def test_complete_fp64_recycle_variants(svt, torch_mod, recycle, over):
    """Recycling only the kept singular vectors, or none (Algorithm 2 every iteration; with
    t = r_max the fixed-rank randomized SVD): identical per-iteration ranks, blocks and
    cooling, and the same completion as the oracle."""
    w = workloads.random_lowrank(300, 250, 8, 0.3, seed=23, n_hold=200, maxit=25)
    ref, got = _run_pair(svt, torch_mod, w, w.maxit, "fp64", recycle=recycle, **over)
    if recycle == "none":
        assert all(e["blocks"] >= 1 for e in ref.log)
    _assert_fp64_parity(w, ref, got)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_complete_mae_stop_and_evaluation_curve(svt, torch_mod, prec):
    """Training-MAE stop rule and the held-out MAE of every iterate (Section 3.2) against
    the oracle: the same stopping iteration and per-iteration held-out MAE."""
    w = workloads.random_lowrank(240, 200, 5, 0.35, seed=29, n_hold=3000, maxit=300)
    tol_mae = 0.05 * float(np.mean(np.abs(w.vals)))
    ev = (w.held_rows, w.held_cols, w.held_vals)
    kw = dict(t=w.t, dt=w.dt, beta=w.beta, eps_thr0=w.eps_thr0, r_max=w.r_max, seed=w.seed,
              n_power=w.n_power, stop="mae")
    ref = oracle.svt(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, tol_mae, w.maxit,
                     eval_set=ev, **kw)
    vals = w.vals if prec == "fp64" else w.vals.astype(np.float32)
    got = svt.complete(w.m, w.n, w.rows, w.cols, vals, w.tau, w.delta, tol_mae, w.maxit,
                       precision=prec, eval_set=(ev[0], ev[1], ev[2] if prec == "fp64" else
                                                 ev[2].astype(np.float32)), **kw)
    assert ref.status == "ok" and 3 < ref.iters < w.maxit
    me_ref = np.array([e["mae_eval"] for e in ref.log])
    me_got = np.array([e["mae_eval"] for e in got.log])
    if prec == "fp64":
        assert got.iters == ref.iters
        assert np.max(np.abs(me_got - me_ref) / me_ref) < 1e-9
    else:
        assert abs(got.iters - ref.iters) <= 1
        n = min(got.iters, ref.iters)
        assert np.max(np.abs(me_got[:n] - me_ref[:n]) / me_ref[:n]) < 1e-3
    assert got.log[-1]["mae"] < tol_mae <= got.log[-2]["mae"]


def test_complete_image1024_mae_stop(svt, torch_mod):
    """The image shape of Section 3.1 at 1024 x 1024 (20% of the pixels, power-law
    spectrum): revealed ranks grow to the 512 cap within 40 iterations, so the eigen start
    runs in its large-r (global-memory Jacobi) form and the CSR-order update takes over
    above 256 columns.  FP64 parity on the first 34 iterations under the training-MAE rule."""
    w = workloads.make("image1024")
    ref, got = _run_pair(svt, torch_mod, w, 34, "fp64", tol=1.0, stop="mae")
    assert max(e["r"] for e in ref.log) > 256
    assert got.iters == ref.iters and got.k == ref.k
    assert [(e["r"], e["k"], e["blocks"]) for e in got.log] == [(e["r"], e["k"], e["blocks"]) for e in ref.log]
    p = ref.pattern
    x_ref = _completed(ref.U, ref.S, ref.V, p.csr_rows(), p.col_idx)
    x_got = _completed(got.U, got.S, got.V, p.csr_rows(), p.col_idx)
    print("image1024 relative difference", _rel(x_got, x_ref))
    assert _rel(x_got, x_ref) < 1e-8


def test_complete_mixed_recycle_kept(svt, torch_mod):
    w = workloads.make("lowrank500")
    ref, got = _run_pair(svt, torch_mod, w, 40, "mixed", recycle="kept")
    p = ref.pattern
    x_obs_ref = _completed(ref.U, ref.S, ref.V, p.csr_rows(), p.col_idx)
    x_obs_got = _completed(got.U, got.S, got.V, p.csr_rows(), p.col_idx)
    assert _rel(x_obs_got, x_obs_ref) < MIXED_TOL


def test_complete_fp64_lowrank500(svt, torch_mod):
    """500x500 rank-10, 20% observed: the full 200-iteration run."""
    w = workloads.small_lowrank()
    ref, got = _run_pair(svt, torch_mod, w, w.maxit, "fp64")
    _assert_fp64_parity(w, ref, got)
    assert got.status == (0 if ref.status == "ok" else 1)


def test_complete_fp64_ratings_scaled(svt, torch_mod):
    """Rating-matrix structure (Zipf rows, empty rows, rank cap) at 0.3 scale."""
    w = workloads.ratings_6040(scale=0.3)
    ref, got = _run_pair(svt, torch_mod, w, 40, "fp64")
    _assert_fp64_parity(w, ref, got)


def test_complete_fp64_power_iterations_and_small_blocks(svt, torch_mod):
    w = workloads.random_lowrank(90, 70, 4, 0.35, seed=11, n_hold=300, maxit=25)
    ref, got = _run_pair(svt, torch_mod, w, 25, "fp64", t=7, dt=3, n_power=1, eps_thr0=0.4)
    _assert_fp64_parity(w, ref, got)


def test_complete_converges_and_recovers(svt, torch_mod):
    w = workloads.random_lowrank(40, 40, 2, 0.6, seed=33, tol=1e-9, maxit=1000)
    w.eps_thr0 = 1e-12
    ref, got = _run_pair(svt, torch_mod, w, w.maxit, "fp64")
    assert got.status == 0 and ref.status == "ok"
    _assert_fp64_parity(w, ref, got)


@pytest.mark.parametrize("name,maxit,kw", [("lowrank500", 60, {}), ("ratings6040", 40, {"scale": 0.3})])
def test_complete_mixed(svt, torch_mod, name, maxit, kw):
    w = workloads.make(name, **kw)
    ref, got = _run_pair(svt, torch_mod, w, maxit, "mixed")
    p = ref.pattern
    x_obs_ref = _completed(ref.U, ref.S, ref.V, p.csr_rows(), p.col_idx)
    x_obs_got = _completed(got.U, got.S, got.V, p.csr_rows(), p.col_idx)
    assert _rel(x_obs_got, x_obs_ref) < MIXED_TOL
    x_h_ref = _completed(ref.U, ref.S, ref.V, w.held_rows, w.held_cols)
    x_h_got = _completed(got.U, got.S, got.V, w.held_rows, w.held_cols)
    assert _rel(x_h_got, x_h_ref) < MIXED_TOL


def test_complete_host_buffers_match_device(svt, torch_mod):
    """The host-pointer path (copies inside the call) gives the device path's result."""
    w = workloads.random_lowrank(120, 90, 3, 0.3, seed=3, n_hold=100, maxit=12)
    kw = dict(t=6, dt=5, eps_thr0=0.6, seed=w.seed)
    host = svt.complete(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, 0.0, 12, **kw)
    dev = svt.complete(w.m, w.n, torch_mod.from_numpy(w.rows).cuda(), torch_mod.from_numpy(w.cols).cuda(),
                       torch_mod.from_numpy(w.vals).cuda(), w.tau, w.delta, 0.0, 12, **kw)
    assert isinstance(host.U, np.ndarray) and host.k == dev.k and host.iters == dev.iters
    assert np.array_equal(host.U, dev.U.cpu().numpy()) and np.array_equal(host.V, dev.V.cpu().numpy())


def test_complete_edge_cases(svt, torch_mod):
    from paper_1704_05528_gb300 import _lib as L
    m, n = 12, 9
    empty = svt.complete(m, n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), 5.0, 1.0,
                         1e-3, 10)
    assert empty.status == L.SVT_OK and empty.k == 0 and empty.iters == 0
    rng = np.random.default_rng(2)
    rows, cols = _coo(rng, m, n, 40)
    vals = rng.standard_normal(40)
    none = svt.complete(m, n, rows, cols, vals, 5.0, 1.0, 1e-3, 0)
    assert none.status == L.SVT_NOT_CONVERGED and none.iters == 0 and none.k == 0
    zero = svt.complete(m, n, rows, cols, np.zeros(40), 5.0, 1.0, 1e-3, 10)
    assert zero.status == L.SVT_OK and zero.k == 0
    bad = vals.copy()
    bad[3] = np.nan
    with pytest.raises(svt.SVTError) as e:
        svt.complete(m, n, rows, cols, bad, 5.0, 1.0, 1e-3, 10)
    assert e.value.status == L.SVT_ERR_NUMERIC
    with pytest.raises(svt.SVTError) as e:
        svt.complete(m, n, rows, np.where(cols == cols[0], n, cols).astype(np.int32), vals, 5.0, 1.0,
                     1e-3, 10)
    assert e.value.status == L.SVT_ERR_INDEX
    dup_r = np.concatenate([rows, rows[:1]])
    dup_c = np.concatenate([cols, cols[:1]])
    with pytest.raises(svt.SVTError) as e:
        svt.complete(m, n, dup_r, dup_c, np.concatenate([vals, vals[:1]]), 5.0, 1.0, 1e-3, 10)
    assert e.value.status == L.SVT_ERR_DUPLICATE
    # tau above every singular value: X stays zero and the residual is 1
    big = svt.complete(m, n, rows, cols, vals, 1e9, 1.0, 1e-3, 3)
    assert big.k == 0 and abs(big.rel_residual - 1.0) < 1e-12


# --------------------------------------------------- full size, bench configuration
@pytest.fixture(scope="module")
def big():
    return workloads.ratings_71567()


def test_full_size_pattern(svt, big):
    _check_pattern(svt, big.m, big.n, big.rows, big.cols)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_first_iterations(svt, torch_mod, big, prec):
    """71,567 x 10,681 with 9.0M observed entries, r_max 100: the first three
    iterations (the initial 100-wide block, then recycled bases) against the oracle."""
    ref, got = _run_pair(svt, torch_mod, big, 3, prec)
    p = ref.pattern
    rng = np.random.default_rng(0)
    sample = rng.choice(p.nnz, size=200_000, replace=False)
    rows_s, cols_s = p.csr_rows()[sample], p.col_idx[sample]
    x_ref = _completed(ref.U, ref.S, ref.V, rows_s, cols_s)
    x_got = _completed(got.U, got.S, got.V, rows_s, cols_s)
    hs = slice(0, 100_000)
    xh_ref = _completed(ref.U, ref.S, ref.V, big.held_rows[hs], big.held_cols[hs])
    xh_got = _completed(got.U, got.S, got.V, big.held_rows[hs], big.held_cols[hs])
    tol = FP64_TOL if prec == "fp64" else MIXED_TOL
    assert _rel(x_got, x_ref) < tol and _rel(xh_got, xh_ref) < tol
    assert got.k == ref.k
    if prec == "fp64":
        assert [e["r"] for e in got.log] == [e["r"] for e in ref.log]
