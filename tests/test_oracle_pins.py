"""Pins for the CPU oracle: each check ties it to something other than itself.

Published known-answer vectors (Philox), brute-force dense scans (pattern),
closed forms (the shrinkage operator of eq. (5) on matrices with a prescribed SVD),
library routines applied to a *different* matrix than the oracle factors (dense SVD
of Y versus the oracle's SVD of the small B), the QB identities of Section 2.2,
Eckart-Young, and exact recovery of small low-rank instances.  The planted-mistake
tests at the end show that plausible bugs in the oracle trip these pins.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats

import oracle
from oracle import fastsvt as osvt
from oracle.philox import philox4x32_10, gaussian_block

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------ Philox
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            words = [int(x, 16) for x in line.split()]
            rows.append((words[:4], words[4:6], words[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox4x32_10(np.array(ctr, dtype=np.uint32), key)
        assert [int(v) for v in got] == want


def test_philox_vectorised_matches_scalar_calls():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x01234567, 0x89ABCDEF)
    batch = philox4x32_10(ctr, key)
    for i in range(0, 64, 7):
        assert np.array_equal(batch[i], philox4x32_10(ctr[i], key))


def test_gaussian_block_distribution():
    g = gaussian_block(1234, 7, 3, 250_000, 4).ravel()
    nsamp = g.size
    assert abs(g.mean()) < 5.0 / math.sqrt(nsamp)
    assert abs(g.var() - 1.0) < 5.0 * math.sqrt(2.0 / nsamp)
    # Kolmogorov-Smirnov against the normal CDF (an independent library routine)
    assert scipy.stats.kstest(g, "norm").pvalue > 1e-4


def test_gaussian_block_layout():
    a = gaussian_block(99, 2, 1, 50, 5)
    b = gaussian_block(99, 2, 1, 50, 6)
    assert np.array_equal(a, b[:, :5])               # odd width drops the last sine
    c = gaussian_block(99, 2, 2, 50, 5)               # another block: other numbers
    assert not np.allclose(a, c)
    d = gaussian_block(99, 3, 1, 50, 5)               # another iteration: other numbers
    assert not np.allclose(a, d)
    # columns 2c and 2c+1 share one counter: g0^2 + g1^2 = -2 ln u1 > 0
    assert np.all(a[:, 0] ** 2 + a[:, 1] ** 2 > 0)
    assert gaussian_block(99, 2, 1, 0, 4).shape == (0, 4)


# ----------------------------------------------------------------------- pattern
def _random_coo(rng, m, n, z):
    flat = rng.choice(m * n, size=z, replace=False)
    return (flat // n).astype(np.int32), (flat % n).astype(np.int32)


@pytest.mark.parametrize("m,n,z", [(7, 5, 12), (1, 9, 4), (9, 1, 5), (13, 17, 0), (20, 30, 200)])
def test_pattern_matches_dense_scan(m, n, z):
    rng = np.random.default_rng(m * 100 + n)
    rows, cols = _random_coo(rng, m, n, z)
    p = oracle.build_pattern(m, n, rows, cols)
    dense = np.zeros((m, n), dtype=bool)
    dense[rows, cols] = True
    r_nz, c_nz = np.nonzero(dense)                    # row-major scan
    assert np.array_equal(p.col_idx, c_nz)
    assert np.array_equal(p.csr_rows(), r_nz)
    assert np.array_equal(p.row_ptr, np.concatenate([[0], np.cumsum(dense.sum(1))]))
    ct_nz, rt_nz = np.nonzero(dense.T)                # column-major scan
    assert np.array_equal(p.row_idx, rt_nz)
    assert np.array_equal(p.col_ptr, np.concatenate([[0], np.cumsum(dense.sum(0))]))
    # perm: CSC slot q holds the same (row, col) as CSR slot perm[q]
    assert np.array_equal(p.csr_rows()[p.perm], rt_nz)
    assert np.array_equal(p.col_idx[p.perm], ct_nz)
    # csr_src: CSR slot k came from COO position csr_src[k]
    assert np.array_equal(rows[p.csr_src], r_nz)
    assert np.array_equal(cols[p.csr_src], c_nz)


def test_pattern_rejects_bad_input():
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_pattern(4, 4, [0, 1, 1], [0, 2, 2])
    assert e.value.kind == "duplicate"
    for rows, cols in (([0, 4], [0, 1]), ([0, 1], [0, 4]), ([-1, 0], [0, 1])):
        with pytest.raises(oracle.OracleError) as e:
            oracle.build_pattern(4, 4, rows, cols)
        assert e.value.kind == "index"
    with pytest.raises(oracle.OracleError):
        oracle.build_pattern(0, 4, [], [])


# ------------------------------------------------------------------ D_tau, eq. (5)
def _householder_orthogonal(rng, k):
    """Orthogonal matrix as a product of k Householder reflectors (no SVD/QR used)."""
    Q = np.eye(k)
    for _ in range(k):
        v = rng.standard_normal(k)
        v /= np.linalg.norm(v)
        Q = Q - 2.0 * np.outer(Q @ v, v)
    return Q


@pytest.mark.parametrize("tau", [0.0, 2.5, 7.0, 100.0])
def test_d_tau_on_prescribed_svd(tau):
    rng = np.random.default_rng(5)
    m, n = 9, 6
    U = _householder_orthogonal(rng, m)[:, :n]
    V = _householder_orthogonal(rng, n)
    s = np.array([11.0, 8.0, 5.5, 3.0, 1.0, 0.25])
    Y = (U * s) @ V.T
    want = (U * np.maximum(s - tau, 0.0)) @ V.T
    assert np.allclose(oracle.d_tau_dense(Y, tau), want, atol=1e-12 * 11.0)


def test_householder_qr_properties():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((40, 7))
    Q, R = oracle.householder_qr(X)
    assert np.allclose(Q.T @ Q, np.eye(7), atol=1e-14)
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, X, atol=1e-13)


def test_spectral_norm_estimate():
    rng = np.random.default_rng(7)
    U = _householder_orthogonal(rng, 30)[:, :4]
    V = _householder_orthogonal(rng, 20)[:, :4]
    Y = sp.csr_matrix((U * np.array([9.0, 3.0, 2.0, 1.0])) @ V.T)
    assert abs(osvt.spectral_norm_estimate(Y, 11, 60) - 9.0) < 1e-10


def test_sampled_product_matches_dense():
    rng = np.random.default_rng(8)
    U, S, V = rng.standard_normal((12, 3)), rng.standard_normal(3), rng.standard_normal((9, 3))
    rows, cols = _random_coo(rng, 12, 9, 30)
    dense = (U * S) @ V.T
    assert np.allclose(oracle.sampled_product(U, S, V, rows, cols), dense[rows, cols],
                       rtol=1e-14, atol=1e-14)


# ----------------------------------------------------------------- R4SVD (Alg. 2/3)
def _sparse_lowrank(rng, m, n, rank, frac):
    M = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    mask = rng.random((m, n)) < frac
    return sp.csr_matrix(np.where(mask, M, 0.0))


@pytest.mark.parametrize("m,n", [(40, 30), (25, 60)])
def test_r4svd_full_precision_equals_dense_svd(m, n):
    rng = np.random.default_rng(m + n)
    Y = _sparse_lowrank(rng, m, n, 5, 0.4)
    Yd = Y.toarray()
    res = oracle.r4svd(Y, None, 1e-15, 1, t=4, dt=3, n_power=0, r_cap=min(m, n), seed=3)
    s_true = np.linalg.svd(Yd, compute_uv=False)
    assert res.r == min(m, n)
    assert np.allclose(res.S, s_true[:res.r], rtol=1e-10, atol=1e-12 * s_true[0])
    # reconstruction: U S V^T reproduces Y
    assert np.allclose((res.U * res.S) @ res.V.T, Yd, atol=1e-10 * s_true[0])


def test_r4svd_qb_identities():
    """Section 2.2, property 1: ||Y - QB||^2 = ||Y||^2 - ||B||^2, and the error
    percentage eps equals the dense residual; property 2: additivity over blocks."""
    rng = np.random.default_rng(12)
    Y = _sparse_lowrank(rng, 60, 45, 8, 0.3)
    Yd = Y.toarray()
    res = oracle.r4svd(Y, None, 0.3, 4, t=5, dt=4, n_power=0, r_cap=45, seed=17)
    Q, Bt = res.Q, res.Bt
    assert np.allclose(Q.T @ Q, np.eye(res.r), atol=1e-13)
    resid = np.linalg.norm(Yd - Q @ Bt.T) ** 2
    nY = np.linalg.norm(Yd) ** 2
    assert abs(resid - (nY - np.linalg.norm(Bt) ** 2)) < 1e-12 * nY
    assert abs(res.eps - resid / nY) < 1e-12
    assert res.eps <= 0.3 < res.eps_trace[-2]           # stopped at the first pass
    # Eckart-Young: no rank-r approximation beats the truncated SVD
    s_true = np.linalg.svd(Yd, compute_uv=False)
    assert res.eps >= np.sum(s_true[res.r:] ** 2) / nY - 1e-12
    # block additivity: the trace decreases by exactly ||B_j||^2/||Y||^2 per block
    widths = [5] + [4] * (len(res.eps_trace) - 2)
    off = 0
    for j, wdt in enumerate(widths):
        blk = np.linalg.norm(Bt[:, off:off + wdt]) ** 2 / nY
        assert abs((res.eps_trace[j] - res.eps_trace[j + 1]) - blk) < 1e-12
        off += wdt


def test_r4svd_recycling_draws_nothing_when_basis_suffices():
    """Algorithm 3: with the exact top-s singular vectors recycled and a threshold
    above their error percentage, no Gaussian block is drawn and the revealed
    singular values are the true top s."""
    rng = np.random.default_rng(21)
    Y = _sparse_lowrank(rng, 50, 40, 4, 0.5)
    Yd = Y.toarray()
    Ut, st, _ = np.linalg.svd(Yd)
    s = 6
    eps_s = np.sum(st[s:] ** 2) / np.sum(st ** 2)
    res = oracle.r4svd(Y, Ut[:, :s], eps_s + 1e-9, 2, t=5, dt=3, n_power=0, r_cap=40, seed=1)
    assert res.blocks == 0 and res.r == s
    assert np.allclose(res.S, st[:s], rtol=1e-12)
    assert abs(res.eps - eps_s) < 1e-12


def test_r4svd_power_iteration_improves_subspace():
    rng = np.random.default_rng(22)
    Y = _sparse_lowrank(rng, 80, 60, 30, 0.5)
    s_true = np.linalg.svd(Y.toarray(), compute_uv=False)
    kw = dict(t=6, dt=6, r_cap=6, seed=9)
    r0 = oracle.r4svd(Y, None, 0.0, 1, n_power=0, **kw)
    r2 = oracle.r4svd(Y, None, 0.0, 1, n_power=2, **kw)
    # Rayleigh-Ritz values are bounded by the true ones; power steps get closer
    assert np.all(r0.S <= s_true[:6] * (1 + 1e-12)) and np.all(r2.S <= s_true[:6] * (1 + 1e-12))
    assert np.sum(s_true[:6] - r2.S) < np.sum(s_true[:6] - r0.S)


@pytest.mark.parametrize("n_power", [0, 2])
def test_r4svd_fixed_rank_is_the_textbook_randomized_svd(n_power):
    """Without a recycled basis and with t = r_cap, R4SVD takes one Gaussian block and is
    the fixed-rank randomized SVD of Section 2.1: X = Y Omega (with power iterations
    X <- Y Y^T X), Q an orthonormal basis of X, B = Q^T Y, SVD of B.  Written out here with
    LAPACK's QR and SVD on the same Omega."""
    rng = np.random.default_rng(41)
    Y = _sparse_lowrank(rng, 90, 70, 12, 0.4)
    T, seed, it = 15, 77, 3
    ro = oracle.r4svd(Y, None, 0.5, it, t=T, dt=4, n_power=n_power, r_cap=T, seed=seed)
    assert (ro.r, ro.blocks) == (T, 1)
    X = Y.toarray() @ gaussian_block(seed, it, 0, Y.shape[1], T)
    for _ in range(n_power):
        X = Y.toarray() @ (Y.toarray().T @ X)
    Q, _ = np.linalg.qr(X)
    Ub, S, Vt = np.linalg.svd(Q.T @ Y.toarray(), full_matrices=False)
    assert np.allclose(ro.S, S, rtol=1e-11, atol=1e-11 * S[0])
    k = 10  # separated part: compare the rank-k reconstructions
    assert np.allclose((ro.U[:, :k] * ro.S[:k]) @ ro.V[:, :k].T, ((Q @ Ub)[:, :k] * S[:k]) @ Vt[:k],
                       atol=1e-10 * S[0])


def test_svt_recycling_variants():
    """Recycling only the kept vectors is recycling all of them when every revealed value is
    kept; without recycling every R4SVD call draws blocks again (Algorithm 2 each time)."""
    rng = np.random.default_rng(8)
    m, n = 70, 60
    M = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n))
    mask = rng.random((m, n)) < 0.5
    rows, cols = np.nonzero(mask)
    kw = dict(t=8, dt=4, eps_thr0=0.05, seed=5, r_max=30)
    runs = {rc: oracle.svt(m, n, rows, cols, M[rows, cols], 1e-9, 1.2, 0.0, 6, recycle=rc, **kw)
            for rc in ("all", "kept", "none")}
    log_all, log_kept = runs["all"].log, runs["kept"].log
    assert all(e["k"] == e["r"] for e in log_all)            # tau below every value
    assert [(e["r"], e["blocks"]) for e in log_kept] == [(e["r"], e["blocks"]) for e in log_all]
    assert np.allclose(runs["kept"].S, runs["all"].S, rtol=1e-12)
    assert all(e["blocks"] >= 1 for e in runs["none"].log)
    assert sum(e["blocks"] for e in runs["none"].log) > sum(e["blocks"] for e in log_all)
    with pytest.raises(oracle.OracleError):
        oracle.svt(m, n, rows, cols, M[rows, cols], 1.0, 1.2, 0.0, 2, recycle="some")


def test_svt_mae_stop_rule_and_evaluation_curve():
    """stop="mae" ends at the first iteration whose training MAE is below tol (Section 3);
    the evaluation-set MAE of each iteration is the mean |A - X| of that iterate on the
    held-out entries, here checked on the returned (last) iterate by a dense product."""
    rng = np.random.default_rng(8)
    m, n = 70, 60
    M = rng.standard_normal((m, 3)) @ rng.standard_normal((3, n))
    mask = rng.random((m, n)) < 0.5
    rows, cols = np.nonzero(mask)
    er, ec = np.nonzero(~mask)
    res = oracle.svt(m, n, rows, cols, M[rows, cols], 5.0, 1.5, 0.05, 200, stop="mae",
                     eval_set=(er, ec, M[er, ec]), seed=3)
    maes = [e["mae"] for e in res.log]
    assert res.status == "ok" and maes[-1] < 0.05 and all(v >= 0.05 for v in maes[:-1])
    X = (res.U * res.S) @ res.V.T
    assert math.isclose(res.log[-1]["mae_eval"], float(np.mean(np.abs(M[er, ec] - X[er, ec]))),
                        rel_tol=1e-12)
    assert math.isclose(res.log[-1]["mae"], float(np.mean(np.abs(M[rows, cols] - X[rows, cols]))),
                        rel_tol=1e-12)
    plain = oracle.svt(m, n, rows, cols, M[rows, cols], 5.0, 1.5, 0.05, 200, seed=3)
    assert all(math.isnan(e["mae_eval"]) for e in plain.log)
    assert plain.log[-1]["rel_residual"] < 0.05 <= plain.log[-2]["rel_residual"]


def test_r4svd_rank_cap_and_exhaustion():
    rng = np.random.default_rng(23)
    # rank-3 matrix with a full pattern: the range is exhausted after 3 directions
    M = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 20))
    Y = sp.csr_matrix(M)
    res = oracle.r4svd(Y, None, 0.0, 1, t=3, dt=2, n_power=0, r_cap=20, seed=2)
    assert res.exhausted and res.r == 3
    assert np.allclose(res.S, np.linalg.svd(M, compute_uv=False)[:3], rtol=1e-10)
    capped = oracle.r4svd(_sparse_lowrank(rng, 30, 20, 10, 0.6), None, 0.0, 1, t=4, dt=3,
                          n_power=0, r_cap=9, seed=2)
    assert capped.r == 9                                  # last block is narrower


# ---------------------------------------------------------------- SVT (Alg. 4)
def _lowrank_problem(seed, m, n, rank, frac):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    rows, cols = _random_coo(rng, m, n, int(frac * m * n))
    return M, rows, cols, M[rows, cols]


def test_svt_recovers_low_rank_matrix():
    """Exact completion of a rank-2 matrix from 60% of its entries (eq. (2)-(3)).

    Square, so that a basis capped at min(m, n) columns is complete and the
    driven-to-zero threshold makes every partial SVD exact."""
    m, n = 40, 40
    M, rows, cols, vals = _lowrank_problem(33, m, n, 2, 0.6)
    res = oracle.svt(m, n, rows, cols, vals, tau=5 * math.sqrt(m * n), delta=1.2 / 0.6,
                     tol=1e-9, maxit=1000, eps_thr0=1e-12, seed=4)
    assert res.status == "ok" and res.k == 2
    X = (res.U * res.S) @ res.V.T
    assert np.linalg.norm(X - M) / np.linalg.norm(M) < 1e-7


def _dense_svt(m, n, rows, cols, vals, tau, delta, iters, k0):
    """Plain full-SVD SVT (eq. (4)-(5)): the SVT-full-SVD comparison method."""
    Y = np.zeros((m, n))
    Y[rows, cols] = k0 * delta * vals
    out = []
    for _ in range(iters):
        X = oracle.d_tau_dense(Y, tau)
        out.append(X[rows, cols].copy())
        R = np.zeros((m, n))
        R[rows, cols] = vals - X[rows, cols]
        Y = Y + delta * R
    return out


def test_svt_with_exact_partial_svd_equals_full_svd_svt():
    """With the threshold driven to zero R4SVD reveals the whole spectrum, so the
    fast SVT iterates must equal those of SVT with a full SVD (square: the capped
    basis spans the whole column space)."""
    m, n = 22, 22
    M, rows, cols, vals = _lowrank_problem(41, m, n, 3, 0.5)
    tau, delta = 3.0 * math.sqrt(m * n), 1.5
    iters = 12
    res = oracle.svt(m, n, rows, cols, vals, tau, delta, tol=0.0, maxit=iters,
                     eps_thr0=1e-14, beta=0.95, seed=8, keep_history=True)
    ref = _dense_svt(m, n, rows, cols, vals, tau, delta, iters, res.k0)
    p = res.pattern
    # the oracle's final X on Lambda (CSR order) versus the dense loop's
    x_final = oracle.sampled_product(res.U, res.S, res.V, p.csr_rows(), p.col_idx)
    dense_final = ref[-1][p.csr_src]
    assert np.allclose(x_final, dense_final, rtol=1e-9, atol=1e-9 * np.abs(dense_final).max())
    assert all(e["r"] == min(m, n) for e in res.log)


def test_svt_initialisation_k0():
    """k0 = ceil(tau / (delta ||P_Lambda A||_2)): the first Y has spectral norm at
    least tau and one fewer step of delta*A would stay below it."""
    m, n = 30, 30
    M, rows, cols, vals = _lowrank_problem(51, m, n, 2, 0.4)
    tau, delta = 200.0, 1.3
    res = oracle.svt(m, n, rows, cols, vals, tau, delta, tol=0.0, maxit=1, seed=2)
    A = np.zeros((m, n))
    A[rows, cols] = vals
    s2 = np.linalg.norm(A, 2)
    assert abs(res.spec_norm - s2) < 1e-8 * s2
    assert res.k0 * delta * s2 >= tau > (res.k0 - 1) * delta * s2


def test_svt_invariants_and_logs():
    m, n = 60, 50
    M, rows, cols, vals = _lowrank_problem(61, m, n, 3, 0.3)
    res = oracle.svt(m, n, rows, cols, vals, 5 * math.sqrt(m * n), 1.2 / 0.3, tol=0.0,
                     maxit=40, eps_thr0=0.8, t=4, dt=3, seed=5)
    ranks = [e["r"] for e in res.log]
    assert all(b >= a for a, b in zip(ranks, ranks[1:]))          # recycling keeps r
    for e in res.log:
        assert e["k"] <= e["r"] <= min(m, n)
        assert e["eps"] <= e["eps_thr"] or e["r"] == min(m, n) or e["exhausted"]
    # cooling: eps_thr shrinks by beta exactly when the residual fails to improve
    for a, b in zip(res.log, res.log[1:]):
        want = a["eps_thr"] * (0.95 if a["cooled"] else 1.0)
        assert abs(b["eps_thr"] - want) < 1e-15
        assert b["cooled"] == (b["rel_residual"] >= a["eps_min"])


def test_svt_edge_cases():
    m, n = 10, 8
    empty = oracle.svt(m, n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), 5.0,
                       1.0, 1e-3, 10)
    assert empty.status == "ok" and empty.k == 0 and empty.iters == 0
    M, rows, cols, vals = _lowrank_problem(71, m, n, 1, 0.5)
    none = oracle.svt(m, n, rows, cols, vals, 1.0, 1.0, 1e-3, 0)
    assert none.status == "not_converged" and none.iters == 0
    zero = oracle.svt(m, n, rows, cols, np.zeros_like(vals), 1.0, 1.0, 1e-3, 10)
    assert zero.status == "ok" and zero.k == 0
    with pytest.raises(oracle.OracleError):
        oracle.svt(m, n, rows, cols, np.where(np.arange(vals.size) == 0, np.nan, vals),
                   1.0, 1.0, 1e-3, 10)
    with pytest.raises(oracle.OracleError):
        oracle.svt(m, n, rows, cols, vals, -1.0, 1.0, 1e-3, 10)


# --------------------------------------------------------- planted mistakes
def test_planted_update_sign_breaks_recovery(monkeypatch):
    """Flip the sign of the P_Lambda(A - X) step: the recovery pin must fail."""
    m, n = 30, 30
    M, rows, cols, vals = _lowrank_problem(81, m, n, 1, 0.5)
    orig = osvt.sampled_product
    monkeypatch.setattr(osvt, "sampled_product",
                        lambda U, S, V, r, c, chunk=1 << 20: 2 * vals_csr_holder[0] - orig(U, S, V, r, c))
    p = oracle.build_pattern(m, n, rows, cols)
    vals_csr_holder = [vals[p.csr_src]]
    res = oracle.svt(m, n, rows, cols, vals, 5 * m, 2.0, tol=1e-6, maxit=200, eps_thr0=1e-12)
    X = (res.U * res.S) @ res.V.T
    assert not (res.status == "ok" and np.linalg.norm(X - M) / np.linalg.norm(M) < 1e-4)


def test_planted_transposed_operand_breaks_qb_identity():
    """Use Y Q instead of Y^T Q for B^T on a square matrix: the QB pin must fail."""
    rng = np.random.default_rng(91)
    Y = _sparse_lowrank(rng, 30, 30, 6, 0.4)
    res = oracle.r4svd(Y, None, 0.2, 1, t=4, dt=3, n_power=0, r_cap=30, seed=3)
    wrong_Bt = np.asarray(Y @ res.Q)
    Yd = Y.toarray()
    nY = np.linalg.norm(Yd) ** 2
    assert abs(np.linalg.norm(Yd - res.Q @ wrong_Bt.T) ** 2 - (nY - np.linalg.norm(wrong_Bt) ** 2)) > 1e-6 * nY


def test_planted_missing_shift_breaks_d_tau():
    """Keep sigma_j > tau without subtracting tau: the prescribed-SVD pin must fail."""
    rng = np.random.default_rng(5)
    U = _householder_orthogonal(rng, 6)
    V = _householder_orthogonal(rng, 6)
    s = np.array([9.0, 7.0, 5.0, 3.0, 2.0, 1.0])
    Y = (U * s) @ V.T
    Uy, sy, Vty = np.linalg.svd(Y)
    keep = sy > 2.5
    wrong = (Uy[:, keep] * sy[keep]) @ Vty[keep]
    want = (U * np.maximum(s - 2.5, 0)) @ V.T
    assert not np.allclose(wrong, want, atol=1e-6)


# ------------------------------------------------- derivatives of unrolled SVT
@pytest.mark.parametrize("m,n", [(9, 7), (6, 8), (10, 10)])
def test_d_tau_jvp_matches_finite_differences(m, n):
    """The full-SVD derivative of D_tau against central differences of eq. (5)."""
    rng = np.random.default_rng(m * 10 + n)
    Y = 3.0 * rng.standard_normal((m, n))
    Z, Z2 = rng.standard_normal((m, n)), rng.standard_normal((m, n))
    tau, h = 2.0, 1e-6
    fd = (oracle.d_tau_dense(Y + h * Z, tau) - oracle.d_tau_dense(Y - h * Z, tau)) / (2 * h)
    J = oracle.d_tau_jvp_dense(Y, tau, Z)
    assert np.linalg.norm(J - fd) < 1e-7 * np.linalg.norm(fd)
    # D_tau is a proximal map, so its Jacobian is symmetric
    assert abs(np.sum(J * Z2) - np.sum(Z * oracle.d_tau_jvp_dense(Y, tau, Z2))) < 1e-12
    fdt = (oracle.d_tau_dense(Y, tau + h) - oracle.d_tau_dense(Y, tau - h)) / (2 * h)
    assert np.linalg.norm(oracle.d_tau_dtau_dense(Y, tau) - fdt) < 1e-7


def test_d_tau_jvp_kept_block_closed_form():
    """On the kept/kept block: (1 - tau/(s_i+s_j)) Zhat_ij + tau/(s_i+s_j) Zhat_ji."""
    rng = np.random.default_rng(3)
    U = _householder_orthogonal(rng, 6)
    V = _householder_orthogonal(rng, 6)
    s = np.array([9.0, 7.0, 5.0, 3.0, 2.0, 1.0])
    Y = (U * s) @ V.T
    Z = rng.standard_normal((6, 6))
    tau = 4.0
    dF = U.T @ oracle.d_tau_jvp_dense(Y, tau, Z) @ V
    Zh = U.T @ Z @ V
    for i in range(3):
        for j in range(3):
            c = tau / (s[i] + s[j])
            want = Zh[i, i] if i == j else (1 - c) * Zh[i, j] + c * Zh[j, i]
            assert abs(dF[i, j] - want) < 1e-12
    assert np.allclose(dF[3:, 3:], 0.0, atol=1e-12)  # complement/complement block vanishes


def test_unrolled_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    m, n = 30, 25
    M = rng.standard_normal((m, 2)) @ rng.standard_normal((2, n))
    flat = rng.choice(m * n, size=300, replace=False)
    rows, cols, vals = flat // n, flat % n, M[flat // n, flat % n]
    hflat = rng.choice(np.setdiff1d(np.arange(m * n), flat), size=50, replace=False)
    hr, hc = hflat // n, hflat % n
    tau, delta, T = 20.0, 1.5, 6
    r = oracle.svt_unrolled_grad(m, n, rows, cols, vals, hr, hc, M[hr, hc], tau, delta, T)

    def f(v=vals, t=tau, d=delta):
        return oracle.svt_unrolled_grad(m, n, rows, cols, v, hr, hc, M[hr, hc], t, d, T, k0=r.k0,
                                        with_grad=False).loss
    h = 1e-5
    assert abs(r.grad_tau - (f(t=tau + h) - f(t=tau - h)) / (2 * h)) < 1e-7 * max(1, abs(r.grad_tau))
    assert abs(r.grad_delta - (f(d=delta + h) - f(d=delta - h)) / (2 * h)) < 1e-7 * max(1, abs(r.grad_delta))
    direction = rng.standard_normal(vals.shape)
    fd = (f(v=vals + h * direction) - f(v=vals - h * direction)) / (2 * h)
    assert abs(np.dot(r.grad_vals, direction) - fd) < 1e-7 * max(1, abs(fd))
