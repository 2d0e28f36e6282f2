"""Writes ratings71567_oracle_300.txt: the binary64 oracle's whole 300-iteration solve of the
71,567 x 10,681 rating workload, reduced to what a test can hold.

The file holds, per iteration, the revealed rank r, the kept count k, the number of new
blocks and the relative residual of Algorithm 4, and the completed matrix
X = U diag(S) V^T of the last iterate at 2,000 observed and 2,000 held-out entries drawn
with a fixed seed.  A whole oracle solve of this workload takes tens of minutes, too long
for a test run; the GPU test compares its own 300-iteration solve with this record.

Only the oracle and the seeded workload generator are used.  Run from the repository
root:  python tests/golden/make_ratings71567_reference.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ratings71567_oracle_300.txt")
N_SAMPLE = 2000
SAMPLE_SEED = 20240


def main():
    w = workloads.make("ratings71567")
    t0 = time.time()
    res = oracle.svt(w.m, w.n, w.rows, w.cols, w.vals, w.tau, w.delta, w.tol, w.maxit,
                     t=w.t, dt=w.dt, n_power=w.n_power, beta=w.beta, eps_thr0=w.eps_thr0,
                     r_max=w.r_max, seed=w.seed)
    seconds = time.time() - t0
    rng = np.random.default_rng(SAMPLE_SEED)
    pick_o = np.sort(rng.choice(w.rows.size, size=N_SAMPLE, replace=False))
    pick_h = np.sort(rng.choice(w.held_rows.size, size=N_SAMPLE, replace=False))
    ro, co = w.rows[pick_o], w.cols[pick_o]
    rh, ch = w.held_rows[pick_h], w.held_cols[pick_h]
    xo = oracle.sampled_product(res.U, res.S, res.V, ro, co)
    xh = oracle.sampled_product(res.U, res.S, res.V, rh, ch)
    with open(OUT, "w") as f:
        f.write("# Binary64 oracle (oracle.svt) on workloads.make('ratings71567'): 71,567 x 10,681,\n")
        f.write(f"# 9,000,049 training ratings, tau = {w.tau!r}, delta = {w.delta!r}, r_max = {w.r_max},\n")
        f.write(f"# maxit = {w.maxit}, tol = {w.tol}; written by tests/golden/make_ratings71567_reference.py\n")
        f.write(f"# ({seconds:.0f} s).  iters {res.iters} k {res.k} k0 {res.k0}\n")
        f.write("# log: iteration r k blocks rel_residual\n")
        for e in res.log:
            f.write(f"log {e['i']} {e['r']} {e['k']} {e['blocks']} {e['rel_residual']!r}\n")
        f.write(f"# last iterate at {N_SAMPLE} observed and {N_SAMPLE} held-out entries (seed {SAMPLE_SEED}):\n")
        f.write("# kind row col x\n")
        for r, c, x in zip(ro, co, xo):
            f.write(f"obs {r} {c} {x!r}\n")
        for r, c, x in zip(rh, ch, xh):
            f.write(f"held {r} {c} {x!r}\n")
    print(f"wrote {OUT} in {seconds:.0f} s")


if __name__ == "__main__":
    main()
