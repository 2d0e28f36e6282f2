"""Seeded generators for the synthetic matrix-completion workloads.

Every generator is a pure function of its seed (numpy PCG64).  Index arrays are
int32, values float64 (callers cast to float32 for the mixed-precision path).
Observed entries come out in a random order: building the sorted pattern is the
solver's job, not the generator's.

Parameter rules (Section 3): tau = ||P_Lambda(A)||_F and delta = sqrt(m*n/ns) where a
workload does not fix them; t = floor(0.05*min(m,n)), dt = 10, beta = 0.95.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Workload:
    name: str
    m: int
    n: int
    rows: np.ndarray          # observed (training) entries, int32
    cols: np.ndarray
    vals: np.ndarray          # float64
    held_rows: np.ndarray     # held-out entries for evaluation, int32
    held_cols: np.ndarray
    held_vals: np.ndarray
    tau: float
    delta: float
    tol: float
    maxit: int
    eps_thr0: float = 0.9
    r_max: int = 0            # 0: no cap beyond min(m, n)
    t: int = -1               # -1: floor(0.05*min(m,n))
    dt: int = 10
    n_power: int = 0
    beta: float = 0.95
    seed: int = 0x5EED
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])

    def options(self) -> dict:
        return dict(t=self.t, dt=self.dt, n_power=self.n_power, beta=self.beta,
                    eps_thr0=self.eps_thr0, r_max=self.r_max, seed=self.seed)


def _split_entries(rng, m, n, flat_obs, vals_fn, n_hold_unobserved=0, frac_hold=0.0):
    """Split observed flat indices into train / held-out and evaluate values."""
    flat_obs = np.asarray(flat_obs, dtype=np.int64)
    if frac_hold > 0.0:
        n_hold = int(round(frac_hold * flat_obs.shape[0]))
        order = rng.permutation(flat_obs.shape[0])
        held = flat_obs[order[:n_hold]]
        train = flat_obs[order[n_hold:]]
    else:
        train = flat_obs
        held = np.zeros(0, dtype=np.int64)
    if n_hold_unobserved > 0:
        mask = np.zeros(m * n, dtype=bool)
        mask[flat_obs] = True
        cand = np.flatnonzero(~mask)
        extra = rng.choice(cand, size=min(n_hold_unobserved, cand.shape[0]), replace=False)
        held = np.concatenate([held, extra])
    tr_r, tr_c = (train // n).astype(np.int32), (train % n).astype(np.int32)
    ho_r, ho_c = (held // n).astype(np.int32), (held % n).astype(np.int32)
    return tr_r, tr_c, vals_fn(tr_r, tr_c), ho_r, ho_c, vals_fn(ho_r, ho_c)


def _factor_values(U, V, scale=1.0):
    def f(r, c):
        out = np.empty(r.shape[0], dtype=np.float64)
        step = 1 << 20
        for s in range(0, r.shape[0], step):
            out[s:s + step] = np.einsum("ij,ij->i", U[r[s:s + step]], V[c[s:s + step]]) * scale
        return out
    return f


def random_lowrank(m, n, rank, frac, seed=0, n_hold=0, tau=None, delta=None, tol=1e-4,
                   maxit=200, **opts) -> Workload:
    """M = U V^T with U, V i.i.d. N(0,1); a uniformly random fraction `frac` observed.

    tau defaults to 5*sqrt(m*n) and delta to 1.2/frac (the usual SVT choices).
    """
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((n, rank))
    z = int(round(frac * m * n))
    flat = rng.choice(m * n, size=z, replace=False)
    r, c, v, hr, hc, hv = _split_entries(rng, m, n, flat, _factor_values(U, V),
                                         n_hold_unobserved=n_hold)
    w = Workload(
        name=f"lowrank_{m}x{n}_r{rank}", m=m, n=n, rows=r, cols=c, vals=v,
        held_rows=hr, held_cols=hc, held_vals=hv,
        tau=5.0 * math.sqrt(m * n) if tau is None else tau,
        delta=1.2 / frac if delta is None else delta, tol=tol, maxit=maxit,
        seed=seed + 0x5EED)
    for k, val in opts.items():
        setattr(w, k, val)
    return w


def small_lowrank(seed=1) -> Workload:
    """500x500, M = U V^T with U, V 500x10 N(0,1); 20% observed uniformly at random.

    tau = 5*sqrt(m*n) = 2500, delta = 1.2/0.2 = 6, stop at relative residual 1e-4
    or 200 iterations.  5,000 unobserved entries are kept for held-out error.
    """
    w = random_lowrank(500, 500, 10, 0.2, seed=seed, n_hold=5000, tol=1e-4, maxit=200)
    w.name = "lowrank_500x500_r10_p0.2"
    return w


def image_512(seed=2) -> Workload:
    """512x512 image-shaped matrix with a power-law spectrum, 50% of pixels observed.

    A = clip(U diag(s) V^T, 0, 255) + N(0,1) noise, s_k = 255 * k^-1.5, U and V Haar
    orthonormal (QR of a Gaussian matrix with the signs of R's diagonal folded in).
    tau = 5*sqrt(m*n) = 2560, tol 1e-3.  The step 1.2/p = 2.4 is capped at 1.9, as for the
    rating workloads: this iterate is not low rank (the noise fills the spectrum), and
    with a step of 2 or more the iteration is not contractive; at 2.4 the relative residual
    swings between 0.5 and 1.8 and stalls at 0.58, and differences at the rounding level
    grow until two binary64 evaluations in different summation orders part by 4e-3 after
    500 iterations.  At 1.9 the residual falls steadily (0.017 after 500 iterations).
    """
    rng = np.random.default_rng(seed)
    m = n = 512

    def haar(k):
        g = rng.standard_normal((k, k))
        q, rr = np.linalg.qr(g)
        return q * np.sign(np.diag(rr))[None, :]

    U, V = haar(m), haar(n)
    s = 255.0 * np.arange(1, m + 1, dtype=np.float64) ** -1.5
    M = np.clip((U * s[None, :]) @ V.T, 0.0, 255.0) + rng.standard_normal((m, n))
    z = (m * n) // 2
    flat = rng.choice(m * n, size=z, replace=False)

    def vals(r, c):
        return M[r, c].astype(np.float64)

    r, c, v, hr, hc, hv = _split_entries(rng, m, n, flat, vals, n_hold_unobserved=10000)
    return Workload(name="image_512x512_p0.5", m=m, n=n, rows=r, cols=c, vals=v,
                    held_rows=hr, held_cols=hc, held_vals=hv,
                    tau=5.0 * math.sqrt(m * n), delta=min(1.2 / 0.5, 1.9), tol=1e-3, maxit=500,
                    seed=seed + 0x5EED)


def image_square(size=8192, seed=6, frac=0.2, rank=1024, decay=1.0) -> Workload:
    """size x size image-shaped matrix with a power-law spectrum, `frac` of pixels observed
    uniformly at random: the shape of the paper's 8192 x 8192 recovery (Section 3.1, 20% of
    the pixels, 13.4M samples).

    A = clip(U diag(s) V^T, 0, 255) + N(0,1) noise with s_k = 255 (size / 16) k^-decay for
    k <= rank (entries of the leading component of order 100), U and V orthonormal (QR of Gaussian size x rank blocks, signs of R's diagonal
    folded in).  Parameter rules of Section 3: tau = ||P_Lambda(A)||_F, delta =
    sqrt(m n / ns); t = floor(0.05 size), dt = 10, r_max = 512, and the stop rule of the
    paper's image runs (training MAE below 1.0) belongs to the caller.
    """
    rng = np.random.default_rng(seed)
    m = n = size

    def basis(k):
        g = rng.standard_normal((size, k))
        q, rr = np.linalg.qr(g)
        return q * np.sign(np.diag(rr))[None, :]

    rank = min(rank, size)
    U, V = basis(rank), basis(rank)
    sv = 255.0 * (size / 16.0) * np.arange(1, rank + 1, dtype=np.float64) ** -float(decay)
    M = (U * sv[None, :]) @ V.T
    np.clip(M, 0.0, 255.0, out=M)
    M += rng.standard_normal((m, n))
    z = int(round(frac * m * n))
    flat = rng.choice(m * n, size=z, replace=False)

    def vals(r, c):
        return M[r, c].astype(np.float64)

    r, c, v, hr, hc, hv = _split_entries(rng, m, n, flat, vals, n_hold_unobserved=100000)
    tau = float(np.sqrt(np.sum(v * v)))
    return Workload(name=f"image_{size}x{size}_p{frac:g}", m=m, n=n, rows=r, cols=c, vals=v,
                    held_rows=hr, held_cols=hc, held_vals=hv, tau=tau,
                    delta=math.sqrt(m * n / r.shape[0]), tol=1e-3, maxit=300, r_max=512,
                    seed=seed + 0x5EED)


def _zipf_weights(rng, k, s):
    """Zipf(s) weights over a random permutation of k items."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    return w[rng.permutation(k)]


def _waterfill_counts(weights, total, cap, floor):
    """Integer counts >= floor, <= cap, proportional to weights, summing to total."""
    k = weights.shape[0]
    counts = np.full(k, floor, dtype=np.int64)
    remaining = total - counts.sum()
    if remaining < 0 or total > cap * k:
        raise ValueError("infeasible count targets")
    open_ = counts < cap
    while remaining > 0:
        w = np.where(open_, weights, 0.0)
        share = w / w.sum() * remaining
        add = np.floor(share).astype(np.int64)
        add = np.minimum(add, cap - counts)
        if add.sum() == 0:
            # hand out the last few one by one, largest weight first among open rows
            order = np.argsort(-np.where(open_, weights, -1.0), kind="stable")
            for i in order[:remaining]:
                if counts[i] < cap:
                    counts[i] += 1
            remaining = total - counts.sum()
        else:
            counts += add
            remaining -= int(add.sum())
        open_ = counts < cap
    return counts


def _sample_cols_without_replacement(rng, counts, col_weights, n):
    """For each row i draw counts[i] distinct columns, successive weighted sampling.

    Rows with more than n/8 entries use exponential-race keys (Efraimidis-Spirakis:
    the counts[i] smallest Exp(1)/w_j).  The other rows draw with replacement in
    sequence and keep the first counts[i] distinct columns in draw order (the same
    law as successive sampling without replacement); rows whose draws run short are
    drawn again with more oversampling.  Returns flat (row*n + col) int64 indices.
    """
    m = counts.shape[0]
    p = col_weights / col_weights.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    big = np.flatnonzero(counts > max(n // 8, 16))
    out = []
    logw = np.log(col_weights)
    chunk = max(1, (1 << 24) // max(n, 1))
    for s in range(0, big.shape[0], chunk):
        rows = big[s:s + chunk]
        keys = np.log(rng.exponential(size=(rows.shape[0], n))) - logw[None, :]
        for t, i in enumerate(rows):
            c = counts[i]
            if c >= n:
                sel = np.arange(n, dtype=np.int64)
            else:
                sel = np.argpartition(keys[t], c - 1)[:c].astype(np.int64)
            out.append(i * np.int64(n) + sel)
    todo = np.flatnonzero((counts <= max(n // 8, 16)) & (counts > 0)).astype(np.int64)
    factor = 1.5
    while todo.size:
        c = counts[todo]
        draws = np.ceil(factor * c + 8).astype(np.int64)
        row_of = np.repeat(todo, draws)
        col = np.searchsorted(cdf, rng.random(row_of.shape[0]), side="right").clip(0, n - 1)
        order = np.arange(row_of.shape[0], dtype=np.int64)       # draw order (rows contiguous)
        key = row_of * n + col
        srt = np.lexsort((order, key))                            # by key, then draw order
        first = np.ones(srt.shape[0], dtype=bool)
        first[1:] = key[srt][1:] != key[srt][:-1]
        keep = np.sort(srt[first])                                # first occurrences, draw order
        kr = row_of[keep]
        # rank of each kept draw within its row
        starts = np.flatnonzero(np.r_[True, kr[1:] != kr[:-1]])
        rank = np.arange(kr.shape[0]) - np.repeat(starts, np.diff(np.r_[starts, kr.shape[0]]))
        need = np.zeros(m, dtype=np.int64)
        need[todo] = c
        have = np.bincount(kr, minlength=m)
        full = have[todo] >= c
        sel = keep[(rank < need[kr]) & (have[kr] >= need[kr])]
        out.append(key[sel])
        todo = todo[~full]
        factor *= 2.0
    return np.concatenate(out)


def _rating_values(U, V, scale, offset, step, lo, hi):
    base = _factor_values(U, V, scale)

    def f(r, c):
        x = base(r, c) + offset
        return np.clip(np.floor(x / step + 0.5) * step, lo, hi)
    return f


def ratings(seed, m, n, total, rank, *, min_per_row, zipf_cols, offset, step, lo, hi,
            hold_frac=0.1, r_max=100, delta_cap=1.9, tol=1e-2, maxit=300, name=None) -> Workload:
    """Rating matrix with Zipf(1.1) row popularity.

    Row counts are proportional to a Zipf(1.1) weight over a random row permutation,
    at least `min_per_row`, capped at n.  Columns are uniform (zipf_cols False) or
    Zipf(1.1)-weighted, drawn without replacement within a row.  Ratings are a rank
    `rank` model M = U V^T / sqrt(rank) shifted by `offset`, rounded to multiples of
    `step` and clipped to [lo, hi].  A fraction `hold_frac` is held out.

    tau = ||P_Lambda(A)||_F (Section 3 rule).  delta = min(sqrt(m*n/ns), delta_cap):
    the Section 3 step sqrt(m*n/ns) makes the iteration diverge on these heavy-tailed
    rows (its fully observed rows carry the sampling operator's eigenvalue 1, and
    the SVT iteration is only stable for steps below 2), so it is capped.
    """
    rng = np.random.default_rng(seed)
    counts = _waterfill_counts(_zipf_weights(rng, m, 1.1), total, n, min_per_row)
    colw = _zipf_weights(rng, n, 1.1) if zipf_cols else np.ones(n)
    flat = _sample_cols_without_replacement(rng, counts, colw, n)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((n, rank))
    vals = _rating_values(U, V, 1.0 / math.sqrt(rank), offset, step, lo, hi)
    r, c, v, hr, hc, hv = _split_entries(rng, m, n, flat, vals, frac_hold=hold_frac)
    tau = float(np.sqrt(np.sum(v * v)))
    delta = min(math.sqrt(m * n / r.shape[0]), delta_cap)
    return Workload(name=name or f"ratings_{m}x{n}", m=m, n=n, rows=r, cols=c, vals=v,
                    held_rows=hr, held_cols=hc, held_vals=hv, tau=tau, delta=delta,
                    tol=tol, maxit=maxit, r_max=r_max, seed=seed + 0x5EED,
                    extra=dict(delta_paper=math.sqrt(m * n / r.shape[0])))


def ratings_6040(seed=3, scale=1.0) -> Workload:
    """6040x3706 rating matrix with 1,000,209 entries (MovieLens-1M shape).

    At least 20 ratings per row plus a Zipf(1.1) share of the rest, capped at n;
    columns uniform without replacement; integer ratings clip(round(3 + M), 1, 5),
    M rank 10.  10% held out.  `scale` shrinks m, n and the entry count together.
    """
    m, n, total = int(6040 * scale), int(3706 * scale), int(1_000_209 * scale * scale)
    return ratings(seed, m, n, total, 10, min_per_row=20, zipf_cols=False, offset=3.0,
                   step=1.0, lo=1.0, hi=5.0, name=f"ratings_{m}x{n}")


def ratings_71567(seed=4, scale=1.0) -> Workload:
    """71,567x10,681 rating matrix with 10,000,054 entries (MovieLens-10M shape).

    Zipf(1.1) row and column popularity; at least one rating per row, capped at n;
    half-step ratings in [0.5, 5] from a rank-20 model shifted to 3.5.  10% held out,
    rank growth capped at 100.  `scale` shrinks m, n and the entry count together.
    """
    m, n, total = int(71_567 * scale), int(10_681 * scale), int(10_000_054 * scale * scale)
    return ratings(seed, m, n, total, 20, min_per_row=1, zipf_cols=True, offset=3.5,
                   step=0.5, lo=0.5, hi=5.0, name=f"ratings_{m}x{n}")


def unrolled_2000(seed=5) -> Workload:
    """2000x2000 rank-20 Gaussian-factor matrix, 10% observed, 40,000 held-out entries.

    tau = 5*sqrt(m*n) = 10,000, delta = 1.2/0.1 = 12; used for 20 unrolled iterations.
    """
    w = random_lowrank(2000, 2000, 20, 0.1, seed=seed, n_hold=40000, tol=0.0, maxit=20)
    w.name = "unrolled_2000x2000_r20_p0.1"
    return w


WORKLOADS = {
    "lowrank500": small_lowrank,
    "image512": image_512,
    "ratings6040": ratings_6040,
    "ratings71567": ratings_71567,
    "unrolled2000": unrolled_2000,
    "image8192": image_square,
    "image1024": lambda **kw: image_square(size=1024, seed=7, rank=256, **kw),
}


def make(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
