"""The synthetic inputs against their stated recipe (CPU).

Each workload stands in for one of the paper's data sets, so its shape, sampling and value
distribution are part of the measurement: the sizes and entry counts, that Λ is a set
(no repeated entry) and the held-out entries lie outside it, the value ranges, the
parameters τ and δ the solve runs with, and that the same seed gives the same inputs.
"""
import math

import numpy as np
import pytest

import workloads


def _flat(w, rows, cols):
    return rows.astype(np.int64) * w.n + cols.astype(np.int64)


def _check_common(w):
    assert w.rows.dtype == np.int32 and w.cols.dtype == np.int32
    assert w.rows.shape == w.cols.shape == w.vals.shape
    assert w.rows.min() >= 0 and w.rows.max() < w.m and w.cols.min() >= 0 and w.cols.max() < w.n
    train = _flat(w, w.rows, w.cols)
    assert np.unique(train).size == train.size                       # Λ is a set
    if w.held_rows.size:
        held = _flat(w, w.held_rows, w.held_cols)
        assert np.unique(held).size == held.size
        assert np.intersect1d(train, held).size == 0                 # held out of Λ
    assert np.all(np.isfinite(w.vals)) and np.all(np.isfinite(w.held_vals))
    return train


def test_lowrank500_recipe():
    w = workloads.make("lowrank500")
    _check_common(w)
    assert (w.m, w.n, w.nnz, w.held_rows.size) == (500, 500, 50_000, 5_000)
    assert w.tau == pytest.approx(5 * math.sqrt(500 * 500)) and w.delta == pytest.approx(1.2 / 0.2)
    assert (w.tol, w.maxit) == (1e-4, 200)
    # a rank-10 product of N(0,1) factors: entries of variance about 10
    assert 8.0 < float(np.var(w.vals)) < 12.0


def test_image512_recipe():
    w = workloads.make("image512")
    _check_common(w)
    assert (w.m, w.n) == (512, 512) and w.nnz == 512 * 512 // 2
    assert w.tau == pytest.approx(2560.0) and w.delta == pytest.approx(1.9)
    assert (w.tol, w.maxit) == (1e-3, 500)


def test_ratings6040_recipe():
    w = workloads.make("ratings6040")
    _check_common(w)
    assert (w.m, w.n) == (6040, 3706)
    assert w.nnz + w.held_rows.size == 1_000_209 and w.held_rows.size == 100_021
    both = np.concatenate([w.vals, w.held_vals])
    assert set(np.unique(both)) <= {1.0, 2.0, 3.0, 4.0, 5.0}         # whole stars
    per_row = np.bincount(np.concatenate([w.rows, w.held_rows]), minlength=w.m)
    assert per_row.min() >= 20 and per_row.max() <= w.n
    assert w.r_max == 100
    assert w.tau == pytest.approx(float(np.linalg.norm(w.vals)))      # τ = ‖P_Λ A‖_F


def test_ratings71567_recipe_and_seed():
    w = workloads.make("ratings71567")
    _check_common(w)
    assert (w.m, w.n) == (71_567, 10_681)
    assert w.nnz == 9_000_049 and w.nnz + w.held_rows.size == 10_000_054
    assert set(np.unique(w.vals)) <= {0.5 * i for i in range(1, 11)}  # half stars in [0.5, 5]
    assert w.r_max == 100 and w.delta == pytest.approx(1.9)           # δ capped (R15)
    assert w.tau == pytest.approx(float(np.linalg.norm(w.vals)))
    # popular rows and columns (Zipf): the fullest row and column are far above the mean
    rc = np.bincount(w.rows, minlength=w.m)
    cc = np.bincount(w.cols, minlength=w.n)
    assert rc.max() > 50 * rc.mean() and cc.max() > 50 * cc.mean()
    assert rc.max() <= w.n
    # the same seed gives the same inputs
    w2 = workloads.make("ratings71567")
    assert np.array_equal(w.rows, w2.rows) and np.array_equal(w.cols, w2.cols)
    assert np.array_equal(w.vals, w2.vals)


def test_unrolled2000_recipe():
    w = workloads.make("unrolled2000")
    _check_common(w)
    assert (w.m, w.n, w.nnz, w.held_rows.size) == (2000, 2000, 400_000, 40_000)
    assert w.tau == pytest.approx(10_000.0) and w.delta == pytest.approx(12.0)


def test_a_different_seed_gives_different_inputs():
    a = workloads.random_lowrank(200, 150, 3, 0.3, seed=1)
    b = workloads.random_lowrank(200, 150, 3, 0.3, seed=1)
    c = workloads.random_lowrank(200, 150, 3, 0.3, seed=2)
    assert np.array_equal(a.rows, b.rows) and np.array_equal(a.vals, b.vals)
    assert not (np.array_equal(a.rows, c.rows) and np.array_equal(a.cols, c.cols))
