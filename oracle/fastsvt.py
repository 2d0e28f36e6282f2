"""Plain FP64 CPU restatement of fast SVT with R4SVD (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this module.  It follows the paper's algorithms step by
step, in their order and notation, with library routines (sparse matmul, LAPACK
Householder QR and SVD) as single steps and no blocking or fusion:

* eq. (3)-(5): the SVT problem, the Uzawa / linearized-Bregman iteration
  X = D_tau(Y), Y <- Y + delta P_Lambda(A - X), and the shrinkage operator D_tau.
* Section 2.2 / Algorithm 2 (R3SVD): an adaptive QB decomposition grown by
  Gaussian blocks orthogonal to the current basis until the error percentage
  eps = (||Y||_F^2 - ||B||_F^2) / ||Y||_F^2 drops to the threshold.
* Section 2.4 / Algorithm 3 (R4SVD): the same loop started from the previous
  iteration's left singular vectors.
* Section 2.5 / Algorithm 4 (fast SVT): cooling of the precision threshold by beta
  whenever the residual stops decreasing.

Readings of points the paper leaves open (each one is listed with its reason in
the design notes; the CUDA path takes the same readings):

* Residual: the printed eps^(i) = ||P_Lambda(A - Y^(i))|| cannot go to zero (Y is the
  dual variable), so the residual is ||P_Lambda(A - X^(i))||_F / ||P_Lambda(A)||_F,
  computed after D_tau; order per iteration: R4SVD -> residual -> cooling -> stop ->
  update.  The stop test is strict (residual < tol), as printed in Algorithm 4.
* Initialisation (Algorithm 4, printed as a scalar): Y^(0) = k0 * delta * P_Lambda(A) with
  k0 = ceil(tau / (delta ||P_Lambda(A)||_2)); the spectral norm is the estimate after a
  fixed number of power steps from a seeded Gaussian start vector.
* Power iterations: the printed X <- Y X is read as X <- Y (Y^T X).
* QB error: the printed (1 - ||B||^2)/||Y||^2 is read as (||Y||^2 - ||B||^2)/||Y||^2
  (the form used inside Algorithms 2 and 3).
* The basis grows by appending new blocks ([Q, Q'] rather than [Q', Q]); the result
  is order-invariant in exact arithmetic.
* Each new block is orthogonalised against Q twice (X <- X - Q Q^T X, repeated).
* Iteration 1 has no basis to recycle and runs Algorithm 2 with a first block of
  width min(t, r_cap); all r columns of U are recycled into the next iteration.
* Rank cap r_cap = min(m, n, r_max); the loop also ends when the range of Y is
  exhausted (a new block whose QR diagonal falls below 1e-7 of its largest
  unprojected column norm is discarded).
* D_tau keeps sigma_j > tau (equality contributes zero either way); the returned
  factors are those of X^(i) = D_tau(Y^(i)).

Parity unpinned: the cooling decisions of Algorithm 4 (when eps_thr is multiplied by
beta) have no external pin -- no closed form or published trajectory exists -- so they
are checked only for consistency with the rule and against the CUDA path.  Every other
step is pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import time

import numpy as np
import scipy.sparse as sp

from .philox import gaussian_block

EXHAUSTED_REL = 1e-7
POWER_SEED_ITER = 0xFFFFFFFF


class OracleError(ValueError):
    """Raised for invalid inputs; `kind` is one of 'arg', 'index', 'duplicate', 'numeric'."""

    def __init__(self, kind, msg):
        super().__init__(f"{kind}: {msg}")
        self.kind = kind


# --------------------------------------------------------------------------- pattern
@dataclass
class Pattern:
    """The observed set Lambda in two sorted orders (P_Lambda is realised by it).

    CSR: entries sorted by (row, col); csr_src[k] is the input (COO) position of CSR
    slot k.  CSC: entries sorted by (col, row); perm[q] is the CSR slot of CSC slot q.
    """
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    csr_src: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray
    perm: np.ndarray

    @property
    def nnz(self):
        return int(self.col_idx.shape[0])

    def csr_rows(self):
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.row_ptr))


def build_pattern(m, n, rows, cols) -> Pattern:
    """Sort the observed index set; reject out-of-range indices and duplicates
    (Lambda is a set of positions, eq. (1))."""
    if m <= 0 or n <= 0:
        raise OracleError("arg", "m and n must be positive")
    rows = np.asarray(rows, dtype=np.int64).ravel()
    cols = np.asarray(cols, dtype=np.int64).ravel()
    if rows.shape != cols.shape:
        raise OracleError("arg", "rows and cols differ in length")
    if rows.size and (rows.min() < 0 or rows.max() >= m or cols.min() < 0 or cols.max() >= n):
        raise OracleError("index", "index out of range")
    order = np.lexsort((cols, rows))           # primary key row, secondary col
    r_s, c_s = rows[order], cols[order]
    if r_s.size > 1 and np.any((r_s[1:] == r_s[:-1]) & (c_s[1:] == c_s[:-1])):
        raise OracleError("duplicate", "duplicate (row, col) entry")
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r_s, minlength=m))
    perm = np.lexsort((r_s, c_s))              # CSR slots ordered by (col, row)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum(np.bincount(c_s, minlength=n))
    return Pattern(m, n, row_ptr, c_s.astype(np.int64), order.astype(np.int64),
                   col_ptr, r_s[perm].astype(np.int64), perm.astype(np.int64))


def _sparse(p: Pattern, y_csr) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(y_csr, dtype=np.float64), p.col_idx, p.row_ptr),
                         shape=(p.m, p.n))


# ------------------------------------------------------------------ small helpers
def householder_qr(X):
    """Thin QR by LAPACK Householder reflections, signs fixed so diag(R) >= 0."""
    Q, R = np.linalg.qr(X, mode="reduced")
    s = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * s[None, :], R * s[:, None]


def spectral_norm_estimate(Ys, seed, steps):
    """||Y||_2 estimate by `steps` power steps v <- Y^T Y v / ||Y^T Y v|| from a
    seeded Gaussian start (used by the initialisation of Algorithm 4)."""
    n = Ys.shape[1]
    v = gaussian_block(seed, POWER_SEED_ITER, 0, n, 1)[:, 0]
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(steps):
        wv = Ys.T @ (Ys @ v)
        lam = np.linalg.norm(wv)
        if lam == 0.0:
            return 0.0
        v = wv / lam
    return math.sqrt(lam)


def d_tau_dense(Y, tau):
    """Shrinkage operator of eq. (5) on a dense matrix via a full SVD."""
    U, s, Vt = np.linalg.svd(np.asarray(Y, dtype=np.float64), full_matrices=False)
    keep = s > tau
    return (U[:, keep] * (s[keep] - tau)[None, :]) @ Vt[keep, :]


def sampled_product(U, S, V, rows, cols, chunk=1 << 20):
    """Entries (U diag(S) V^T)_{rows[e], cols[e]}, summed over j in increasing order."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    out = np.zeros(rows.shape[0], dtype=np.float64)
    if U.shape[1] == 0:
        return out
    US = U * S[None, :]
    for s0 in range(0, rows.shape[0], chunk):
        out[s0:s0 + chunk] = np.einsum("ij,ij->i", US[rows[s0:s0 + chunk]], V[cols[s0:s0 + chunk]])
    return out


# ------------------------------------------------------------------------- R4SVD
@dataclass
class R4SVDResult:
    U: np.ndarray          # m x r, left singular vectors (Q U_B)
    S: np.ndarray          # r singular values, descending
    V: np.ndarray          # n x r right singular vectors
    r: int                 # revealed rank
    eps: float             # final error percentage
    blocks: int            # Gaussian blocks drawn
    normY2: float
    normB: float
    exhausted: bool
    Q: np.ndarray = None
    Bt: np.ndarray = None
    eps_trace: list = field(default_factory=list)


def r4svd(Ys, U_prev, eps_thr, it, *, t, dt, n_power, r_cap, seed) -> R4SVDResult:
    """Algorithm 3 (R4SVD); with U_prev empty it is Algorithm 2 (R3SVD).

    Ys: m x n sparse Y^(i); U_prev: m x s recycled basis or None.
    Block b of iteration `it` uses Omega = gaussian_block(seed, it, b, n, w).
    """
    m, n = Ys.shape
    normY2 = float(Ys.multiply(Ys).sum())
    eps_of = (lambda nb: (normY2 - nb) / normY2) if normY2 > 0 else (lambda nb: 0.0)
    if U_prev is not None and U_prev.shape[1] > 0:
        Q = np.array(U_prev, dtype=np.float64)             # recycling
        Bt = np.asarray(Ys.T @ Q)                            # B^T = Y^T Q
        normB = float(np.sum(Bt * Bt))
        r = Q.shape[1]
        first = False
    else:
        Q = np.zeros((m, 0))
        Bt = np.zeros((n, 0))
        normB = 0.0
        r = 0
        first = True                                         # R3SVD initial block
    eps = eps_of(normB)
    trace = [eps]
    b = 0
    exhausted = False
    while (first or eps > eps_thr) and r < r_cap:
        w = min(min(t, r_cap) if first else dt, r_cap - r)
        Omega = gaussian_block(seed, it, b, n, w)
        b += 1
        X = np.asarray(Ys @ Omega)
        for _ in range(n_power):                             # power iterations
            X = np.asarray(Ys @ np.asarray(Ys.T @ X))
        scale = float(np.max(np.linalg.norm(X, axis=0))) if w > 0 else 0.0
        if r > 0:
            for _ in range(2):                               # X <- X - Q Q^T X, twice
                X = X - Q @ (Q.T @ X)
        Qn, R = householder_qr(X)
        if scale == 0.0 or np.min(np.abs(np.diag(R))) <= EXHAUSTED_REL * scale:
            exhausted = True
            break
        Btn = np.asarray(Ys.T @ Qn)                          # B' = Q'^T Y, stored transposed
        Q = np.concatenate([Q, Qn], axis=1)
        Bt = np.concatenate([Bt, Btn], axis=1)
        normB += float(np.sum(Btn * Btn))
        eps = eps_of(normB)
        trace.append(eps)
        r += w
        first = False
    if r == 0:
        return R4SVDResult(np.zeros((m, 0)), np.zeros(0), np.zeros((n, 0)), 0, eps, b,
                           normY2, normB, exhausted, Q, Bt, trace)
    Ub, S, Vbt = np.linalg.svd(Bt.T, full_matrices=False)  # svd(B), B = Bt^T (r x n)
    U = Q @ Ub
    return R4SVDResult(U, S, Vbt.T, r, eps, b, normY2, normB, exhausted, Q, Bt, trace)


# --------------------------------------------------------------------------- SVT
@dataclass
class SVTResult:
    U: np.ndarray          # m x k
    S: np.ndarray          # k shrunk singular values sigma_j - tau
    V: np.ndarray          # n x k
    k: int
    iters: int
    rel_residual: float
    status: str            # 'ok' | 'not_converged'
    k0: int
    spec_norm: float
    log: list = field(default_factory=list)
    y_final: np.ndarray = None     # Y^(iters) in CSR order (before the last update)
    pattern: Pattern = None


def svt(m, n, rows, cols, vals, tau, delta, tol, maxit, *, t=-1, dt=10, n_power=0,
        beta=0.95, eps_thr0=0.9, r_max=0, seed=0x5EED, power_steps=100,
        keep_history=False, recycle="all", stop="residual", eval_set=None) -> SVTResult:
    """Algorithm 4 (fast SVT with R4SVD) on the observed entries (rows, cols, vals).

    recycle picks the basis handed to the next R4SVD call (Section 2.3): "all" the r
    revealed left singular vectors (Algorithm 3, the paper's method), "kept" the k above
    tau, "none" no basis (Algorithm 2 every iteration; with t = r_max a fixed-rank
    randomized SVD as in Section 2.1).

    stop="residual" ends when ||P_Lambda(A - X)||_F / ||P_Lambda(A)||_F < tol (Algorithm 4),
    stop="mae" when the mean |A - X| over Lambda < tol (the rule of Section 3).
    eval_set = (rows, cols, vals) of held-out entries: each log entry gets "mae_eval", the
    mean |A - X^(i)| over them (the testing-set curve of Section 3.2)."""
    if not (tau > 0 and delta > 0) or maxit < 0 or dt <= 0 or not (0 < beta < 1):
        raise OracleError("arg", "bad scalar parameter")
    if recycle not in ("all", "kept", "none"):
        raise OracleError("arg", "recycle must be all, kept or none")
    if stop not in ("residual", "mae"):
        raise OracleError("arg", "stop must be residual or mae")
    p = build_pattern(m, n, rows, cols)
    vals = np.asarray(vals, dtype=np.float64).ravel()
    if vals.shape[0] != p.nnz:
        raise OracleError("arg", "vals length differs from rows")
    if not np.all(np.isfinite(vals)):
        raise OracleError("numeric", "non-finite observed value")
    a = vals[p.csr_src]                                     # P_Lambda(A) in CSR order
    t_eff = int(math.floor(0.05 * min(m, n))) if t < 0 else int(t)
    t_eff = max(t_eff, 1)
    r_cap = min(m, n) if r_max <= 0 else min(m, n, r_max)
    nA = float(np.sqrt(np.sum(a * a)))
    empty = SVTResult(np.zeros((m, 0)), np.zeros(0), np.zeros((n, 0)), 0, 0, 0.0, "ok", 0,
                      0.0, [], a.copy(), p)
    if p.nnz == 0 or nA == 0.0:
        return empty
    As = _sparse(p, a)
    s2 = spectral_norm_estimate(As, seed, power_steps)
    k0 = int(math.ceil(tau / (delta * s2))) if s2 > 0.0 else 1
    y = k0 * delta * a                                       # Y^(0) = k0 delta P_Lambda(A)
    eps_thr = float(eps_thr0)
    eps_min = math.inf
    U_prev = None
    rows_csr = p.csr_rows()
    log = []
    res = None
    for i in range(1, maxit + 1):
        t_iter = time.perf_counter()
        Ys = _sparse(p, y)
        rs = r4svd(Ys, U_prev, eps_thr, i, t=t_eff, dt=dt, n_power=n_power, r_cap=r_cap,
                   seed=seed)
        keep = rs.S > tau                                    # D_tau, eq. (5)
        Uk, Sk, Vk = rs.U[:, keep], rs.S[keep] - tau, rs.V[:, keep]
        x = sampled_product(Uk, Sk, Vk, rows_csr, p.col_idx)  # P_Lambda(X^(i))
        d = a - x
        rel = float(np.sqrt(np.sum(d * d))) / nA
        mae = float(np.mean(np.abs(d)))
        mae_eval = math.nan
        if eval_set is not None:                             # held-out MAE of X^(i)
            er, ec, ev = eval_set
            xe = sampled_product(Uk, Sk, Vk, np.asarray(er), np.asarray(ec))
            mae_eval = float(np.mean(np.abs(np.asarray(ev, dtype=np.float64) - xe)))
        entry = dict(i=i, r=rs.r, k=int(keep.sum()), blocks=rs.blocks, eps=rs.eps, mae_eval=mae_eval,
                     eps_thr=eps_thr, rel_residual=rel, mae=mae, exhausted=rs.exhausted,
                     sigma_max=float(rs.S[0]) if rs.r else 0.0,
                     margin_tau=float(np.min(np.abs(rs.S - tau))) if rs.r else math.inf,
                     eps_trace=rs.eps_trace)
        if rel < eps_min:                                    # simulated-annealing cooling
            eps_min = rel
            entry["cooled"] = False
        else:
            eps_thr = beta * eps_thr
            entry["cooled"] = True
        entry["eps_min"] = eps_min
        entry["seconds"] = time.perf_counter() - t_iter
        if keep_history:
            entry["S"] = rs.S.copy()
        log.append(entry)
        res = SVTResult(Uk, Sk, Vk, int(keep.sum()), i, rel, "ok", k0, s2, log, y.copy(), p)
        if (mae if stop == "mae" else rel) < tol:
            return res
        y = y + delta * d                                    # Y <- Y + delta P_Lambda(A - X)
        U_prev = {"all": rs.U, "kept": rs.U[:, keep], "none": None}[recycle]
    if res is None:                                          # maxit == 0
        empty.status = "not_converged"
        return empty
    res.status = "not_converged"
    return res
