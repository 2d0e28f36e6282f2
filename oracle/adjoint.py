"""Reference derivatives for unrolled SVT (test infrastructure only).

The paper defines the SVT iteration X^(i) = D_tau(Y^(i)), Y^(i+1) = Y^(i) + delta
P_Lambda(A - X^(i)) (eq. (4)) with the shrinkage operator D_tau of eq. (5).  Here that
iteration is unrolled for a fixed number of steps and differentiated with respect to
tau, delta and the observed values, for a loss on held-out entries.  Everything is dense
binary64 with full SVDs: slow and direct, as a reference for the adjoint on the GPU.

Derivative of D_tau.  D_tau is the spectral function F(Y) = U diag(f(sigma)) V^T with
f(s) = max(s - tau, 0).  With Y = U Sigma V^T a full SVD and Z_hat = U^T Z V, its
directional derivative is U dF V^T where, for the leading min(m, n) block,
    dF_ii = f'(sigma_i) Z_hat_ii,
    dF_ij = (A_ij + B_ij)/2 Z_hat_ij + (A_ij - B_ij)/2 Z_hat_ji   (i != j),
    A_ij = (f_i - f_j)/(sigma_i - sigma_j),  B_ij = (f_i + f_j)/(sigma_i + sigma_j),
and, on the rectangular remainder, dF_ij = (f_j / sigma_j) Z_hat_ij (extra rows, m > n)
or (f_i / sigma_i) Z_hat_ij (extra columns, n > m).  For i, j both kept this reduces to
dF_ij = (1 - tau/(s_i+s_j)) Z_hat_ij + (tau/(s_i+s_j)) Z_hat_ji.  The map is symmetric,
so it is its own adjoint.  dD_tau/dtau = -U_K V_K^T (K: sigma > tau).

Parity unpinned: nothing here; the JVP is pinned by finite differences of d_tau_dense and
the gradient by central finite differences of the unrolled forward.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

from .fastsvt import build_pattern, spectral_norm_estimate, _sparse


def _svd_full(Y):
    U, s, Vt = np.linalg.svd(np.asarray(Y, dtype=np.float64), full_matrices=True)
    return U, s, Vt.T


def d_tau_jvp_dense(Y, tau, Z, svd=None):
    """Directional derivative of D_tau at Y in direction Z (dense, full SVD)."""
    m, n = Y.shape
    U, s, V = _svd_full(Y) if svd is None else svd
    k = min(m, n)
    f = np.maximum(s - tau, 0.0)
    fp = (s > tau).astype(np.float64)
    Zh = U.T @ Z @ V
    dF = np.zeros((m, n))
    si, sj = s[:, None], s[None, :]
    fi, fj = f[:, None], f[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        A = np.where(np.abs(si - sj) > 0, (fi - fj) / (si - sj), fp[:, None] * np.ones((1, k)))
        B = np.where(si + sj > 0, (fi + fj) / (si + sj), 0.0)
    Zk = Zh[:k, :k]
    blk = 0.5 * (A + B) * Zk + 0.5 * (A - B) * Zk.T
    blk[np.diag_indices(k)] = fp * np.diag(Zk)
    dF[:k, :k] = blk
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(s > 0, f / s, 0.0)
    if m > n:
        dF[n:, :] = Zh[n:, :] * ratio[None, :]
    elif n > m:
        dF[:, m:] = Zh[:, m:] * ratio[:, None]
    return U @ dF @ V.T


def d_tau_dtau_dense(Y, tau, svd=None):
    """dD_tau(Y)/dtau = -U_K V_K^T."""
    U, s, V = _svd_full(Y) if svd is None else svd
    keep = s > tau
    return -(U[:, :len(s)][:, keep] @ V[:, :len(s)][:, keep].T)


@dataclass
class UnrolledResult:
    loss: float
    grad_vals: np.ndarray    # d loss / d vals, in the caller's entry order
    grad_tau: float
    grad_delta: float
    x_held: np.ndarray       # X^(T) on the held-out entries
    k0: int


def svt_unrolled_grad(m, n, rows, cols, vals, held_rows, held_cols, held_vals, tau, delta, T,
                      *, k0=None, seed=0x5EED, power_steps=100, with_grad=True) -> UnrolledResult:
    """Unrolled SVT (eq. (4)-(5)) for T steps with exact D_tau, its held-out loss
    L = mean over H of (X^(T) - A)^2, and dL/dvals, dL/dtau, dL/ddelta.

    Y^(1) = k0 delta P_Lambda(A) (k0 held fixed), X^(i) = D_tau(Y^(i)) for i = 1..T and
    Y^(i+1) = Y^(i) + delta P_Lambda(A - X^(i)) for i < T.
    """
    p = build_pattern(m, n, rows, cols)
    a = np.asarray(vals, dtype=np.float64)[p.csr_src]
    pr, pc = p.csr_rows(), p.col_idx
    if k0 is None:
        s2 = spectral_norm_estimate(_sparse(p, a), seed, power_steps)
        k0 = int(math.ceil(tau / (delta * s2))) if s2 > 0 else 1
    y = k0 * delta * a
    Ys, svds, Xs = [], [], []
    for i in range(1, T + 1):
        Yd = np.zeros((m, n))
        Yd[pr, pc] = y
        sv = _svd_full(Yd)
        U, s, V = sv
        keep = s > tau
        X = (U[:, :len(s)][:, keep] * (s[keep] - tau)) @ V[:, :len(s)][:, keep].T
        Ys.append(Yd)
        svds.append(sv)
        Xs.append(X)
        if i < T:
            y = y + delta * (a - X[pr, pc])
    hr = np.asarray(held_rows, dtype=np.int64)
    hc = np.asarray(held_cols, dtype=np.int64)
    hv = np.asarray(held_vals, dtype=np.float64)
    xh = Xs[-1][hr, hc]
    res = xh - hv
    loss = float(np.mean(res * res)) if hr.size else 0.0
    if not with_grad:
        return UnrolledResult(loss, None, 0.0, 0.0, xh, k0)
    G = np.zeros((m, n))
    np.add.at(G, (hr, hc), 2.0 * res / max(hr.size, 1))
    # through X^(T) = D_tau(Y^(T))
    gtau = float(np.sum(G * d_tau_dtau_dense(Ys[-1], tau, svds[-1])))
    Jg = d_tau_jvp_dense(Ys[-1], tau, G, svds[-1])
    ybar = Jg[pr, pc]                      # dL/dY^(T) on Lambda
    abar = np.zeros_like(a)
    dbar = 0.0
    for i in range(T - 1, 0, -1):          # Y^(i+1) = Y^(i) + delta P(A - X^(i))
        Xi = Xs[i - 1]
        abar += delta * ybar
        dbar += float(np.dot(ybar, a - Xi[pr, pc]))
        Zb = np.zeros((m, n))
        Zb[pr, pc] = ybar
        gtau -= delta * float(np.sum(Zb * d_tau_dtau_dense(Ys[i - 1], tau, svds[i - 1])))
        ybar = ybar - delta * d_tau_jvp_dense(Ys[i - 1], tau, Zb, svds[i - 1])[pr, pc]
    abar += k0 * delta * ybar              # Y^(1) = k0 delta A
    dbar += k0 * float(np.dot(ybar, a))
    grad_vals = np.zeros_like(abar)
    grad_vals[p.csr_src] = abar
    return UnrolledResult(loss, grad_vals, gtau, dbar, xh, k0)
