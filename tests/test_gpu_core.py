"""The dense-row core of the binary32 fused update (tensor cores) against the gather path
and the CPU oracle.

With core_rows > 0 the fullest rows of Lambda are stored as a dense panel, and the update
of eq. (4)-(5) and the recycled product of Algorithm 3 run there as TF32x3 tensor-core
GEMMs; the rest of Lambda stays on the gather kernel.  The two layouts compute the same
binary32-accurate quantities in different orders, so a solve with the core must follow
the solve without it (identical revealed ranks and kept counts, residuals to 1e-5) and
stay within the mixed-precision bar of the binary64 oracle.  The cases cover a core that
is not a whole number of 128-slot tiles, ragged q tiles, kept counts from 0 upwards and
every K chunk count.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt, torch


def _zipf_pattern(rng, m, n, z, heavy_rows, heavy_frac):
    """z distinct entries; `heavy_rows` rows hold about heavy_frac of them (dense core)."""
    heavy = rng.choice(m, size=heavy_rows, replace=False)
    n_heavy = int(heavy_frac * z)
    flat_h = rng.choice(heavy_rows * n, size=min(n_heavy, heavy_rows * n), replace=False)
    rows_h = heavy[flat_h // n]
    cols_h = flat_h % n
    taken = set(zip(rows_h.tolist(), cols_h.tolist()))
    rows, cols = list(rows_h), list(cols_h)
    while len(rows) < z:
        r, c = int(rng.integers(m)), int(rng.integers(n))
        if (r, c) not in taken:
            taken.add((r, c))
            rows.append(r)
            cols.append(c)
    order = rng.permutation(len(rows))
    return np.asarray(rows, np.int32)[order], np.asarray(cols, np.int32)[order]


def _problem(seed, m, n, z, rank, heavy_rows, heavy_frac, n_hold=2000):
    rng = np.random.default_rng(seed)
    rows, cols = _zipf_pattern(rng, m, n, z, heavy_rows, heavy_frac)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((n, rank))
    vals = np.einsum("ij,ij->i", U[rows], V[cols]) / np.sqrt(rank) + 3.0
    hr = rng.integers(0, m, n_hold).astype(np.int32)
    hc = rng.integers(0, n, n_hold).astype(np.int32)
    hv = np.einsum("ij,ij->i", U[hr], V[hc]) / np.sqrt(rank) + 3.0
    return rows, cols, vals, hr, hc, hv


def _completed(res, rows, cols):
    to = lambda t: t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    return oracle.sampled_product(to(res.U), to(res.S), to(res.V), rows, cols)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m,n,z,heavy,core_rows,r_max,t", [
    (1500, 700, 120_000, 150, 150, 60, 20),    # 150 core rows: one full tile and a ragged one
    (1000, 1030, 150_000, 300, 256, 100, 40),  # two full tiles, n not a multiple of 128
    (900, 450, 60_000, 80, 128, 128, 128),     # r = 128: widest core product
    (600, 260, 30_000, 64, 64, 24, 8),         # narrow: r = 24, one K chunk
])
def test_core_follows_the_gather_path_and_the_oracle(env, m, n, z, heavy, core_rows, r_max, t):
    svt, torch = env
    rows, cols, vals, hr, hc, hv = _problem(m + n, m, n, z, 8, heavy, 0.6)
    tau = 0.8 * np.linalg.norm(vals)
    delta = min(np.sqrt(m * n / z), 1.9)
    maxit = 30
    kw = dict(t=t, dt=10, r_max=r_max, eps_thr0=0.9, seed=11)
    d = lambda a: torch.from_numpy(a).cuda()
    v32 = vals.astype(np.float32)
    runs = {}
    for cr in (0, core_rows):
        runs[cr] = svt.complete(m, n, d(rows), d(cols), d(v32), tau, delta, 0.0, maxit,
                                precision="mixed", core_rows=cr, **kw)
    gat, cor = runs[0], runs[core_rows]
    assert [e["r"] for e in cor.log] == [e["r"] for e in gat.log]
    assert [e["k"] for e in cor.log] == [e["k"] for e in gat.log]
    assert max(e["k"] for e in cor.log) > 0
    res_g = np.array([e["rel_residual"] for e in gat.log])
    res_c = np.array([e["rel_residual"] for e in cor.log])
    assert np.max(np.abs(res_c - res_g) / res_g) < 1e-5
    ref = oracle.svt(m, n, rows, cols, vals, tau, delta, 0.0, maxit, **kw)
    p = ref.pattern
    x_ref = _completed(ref, p.csr_rows(), p.col_idx)
    e_core = _rel(_completed(cor, p.csr_rows(), p.col_idx), x_ref)
    e_gath = _rel(_completed(gat, p.csr_rows(), p.col_idx), x_ref)
    e_held = _rel(_completed(cor, hr, hc), _completed(ref, hr, hc))
    print(f"\ncore {core_rows} rows: vs oracle observed {e_core:.2e} (gather path {e_gath:.2e}), "
          f"held-out {e_held:.2e}")
    assert e_core < 1e-3 and e_held < 1e-3


def test_core_with_nothing_kept_and_the_exact_update(env):
    """tau above every singular value: k = 0, X = 0 on the core, and Y must grow by exactly
    delta * A on Lambda each iteration, in the core as in the rest."""
    svt, torch = env
    m, n, z = 700, 300, 40_000
    rows, cols, vals, _, _, _ = _problem(3, m, n, z, 4, 128, 0.7)
    d = lambda a: torch.from_numpy(a).cuda()
    kw = dict(t=16, dt=8, r_max=32, seed=5)
    v32 = vals.astype(np.float32)
    a = svt.complete(m, n, d(rows), d(cols), d(v32), 1e9, 1.0, 0.0, 4, precision="mixed", core_rows=128, **kw)
    b = svt.complete(m, n, d(rows), d(cols), d(v32), 1e9, 1.0, 0.0, 4, precision="mixed", core_rows=0, **kw)
    assert a.k == b.k == 0
    assert [e["r"] for e in a.log] == [e["r"] for e in b.log]
    for ea, eb in zip(a.log, b.log):
        assert abs(ea["rel_residual"] - 1.0) < 1e-12 and abs(eb["rel_residual"] - 1.0) < 1e-12
        assert abs(ea["sigma_max"] - eb["sigma_max"]) <= 1e-5 * eb["sigma_max"]
