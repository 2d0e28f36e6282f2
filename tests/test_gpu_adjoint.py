"""Gradient of unrolled SVT through the C ABI against the FP64 full-SVD reference.

The reference (oracle.svt_unrolled_grad) runs exact SVT with dense full SVDs and
differentiates it in closed form.  The GPU forward evaluates D_tau by R4SVD followed by a
Ritz refinement to a residual bound, so it is exact SVT to that bound and its hand-written
adjoint (kept-block closed form + CG solves for the rest of the spectrum) must give the
reference gradient.  Central finite differences of the GPU forward check the same
gradient without the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def svt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_05528_gb300 as svt
    return svt


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _scalar_close(got, ref, rtol):
    return abs(got - ref) <= rtol * max(abs(ref), 1e-12)


def _call(svt, w, tau, delta, steps, **kw):
    return svt.unrolled_grad(w.m, w.n, w.rows, w.cols, w.vals, w.held_rows, w.held_cols,
                             w.held_vals, tau, delta, steps, seed=w.seed, **kw)


def _reference(w, tau, delta, steps):
    return oracle.svt_unrolled_grad(w.m, w.n, w.rows, w.cols, w.vals, w.held_rows, w.held_cols,
                                    w.held_vals, tau, delta, steps, seed=w.seed)


def _check_against(got, ref, rtol, x_rtol):
    assert got["info"]["k0"] == ref.k0
    assert got["info"]["cg_capped"] == 0
    assert _scalar_close(got["loss"], ref.loss, x_rtol)
    assert _rel(got["x_held"], ref.x_held) <= x_rtol
    assert _rel(got["grad_vals"], ref.grad_vals) <= rtol
    assert _scalar_close(got["grad_tau"], ref.grad_tau, rtol)
    assert _scalar_close(got["grad_delta"], ref.grad_delta, rtol)


# Square, full rank revealed: R4SVD alone is already exact, the refinement has nothing to do.
@pytest.mark.parametrize("steps,ckpt", [(7, 3), (5, 5)])
def test_gradient_full_basis_matches_reference(svt, steps, ckpt):
    w = workloads.random_lowrank(48, 48, 3, 0.4, seed=3, n_hold=300)
    tau, delta = 3.0 * np.sqrt(w.m * w.n), 1.5
    got = _call(svt, w, tau, delta, steps, checkpoint_every=ckpt, cg_tol=1e-13, cg_maxit=2000,
                precision="fp64", eps_thr0=1e-14, t=4, dt=8)
    _check_against(got, _reference(w, tau, delta, steps), 1e-7, 1e-9)


# Hot threshold and a rank cap well below min(m, n): the R4SVD triplets are approximate
# and the Ritz refinement is what makes D_tau exact.
@pytest.mark.parametrize("m,n", [(240, 180), (150, 220)])
def test_gradient_with_refinement_matches_reference(svt, m, n):
    w = workloads.random_lowrank(m, n, 4, 0.3, seed=11, n_hold=600)
    tau, delta, steps = 5.0 * np.sqrt(m * n), 1.2 / 0.3, 8
    got = _call(svt, w, tau, delta, steps, checkpoint_every=3, cg_tol=1e-12, cg_maxit=3000,
                precision="fp64", r_max=40, t=10, dt=10)
    _check_against(got, _reference(w, tau, delta, steps), 1e-6, 1e-8)
    assert got["info"]["ritz_steps"] > 0 and got["info"]["ritz_capped"] == 0, got["info"]
    plain = _call(svt, w, tau, delta, steps, checkpoint_every=3, precision="fp64", r_max=40, t=10,
                  dt=10, ritz_maxit=0)
    assert plain["info"]["ritz_steps"] == 0 and np.isfinite(plain["loss"])


def test_gradient_matches_finite_differences(svt):
    w = workloads.random_lowrank(40, 40, 2, 0.5, seed=5, n_hold=200)
    tau, delta, steps = 2.5 * np.sqrt(w.m * w.n), 1.2, 6
    kw = dict(checkpoint_every=2, cg_tol=1e-13, cg_maxit=2000, precision="fp64")
    g = _call(svt, w, tau, delta, steps, **kw)

    def loss(v=w.vals, t=tau, d=delta):
        return svt.unrolled_grad(w.m, w.n, w.rows, w.cols, v, w.held_rows, w.held_cols, w.held_vals,
                                 t, d, steps, seed=w.seed, with_grad=False, **kw)["loss"]
    h = 1e-4
    fd_tau = (loss(t=tau + h) - loss(t=tau - h)) / (2 * h)
    fd_delta = (loss(d=delta + h) - loss(d=delta - h)) / (2 * h)
    direction = np.random.default_rng(1).standard_normal(w.vals.shape)
    fd_vals = (loss(v=w.vals + h * direction) - loss(v=w.vals - h * direction)) / (2 * h)
    assert _scalar_close(g["grad_tau"], fd_tau, 1e-5)
    assert _scalar_close(g["grad_delta"], fd_delta, 1e-5)
    assert _scalar_close(float(np.dot(g["grad_vals"], direction)), fd_vals, 1e-5)


def test_forward_only_and_uncertified_kept_set(svt):
    w = workloads.random_lowrank(60, 50, 3, 0.4, seed=9, n_hold=100)
    tau, delta = 2.0 * np.sqrt(w.m * w.n), 1.5
    # a first block of one column: the kept set is certified only after the basis grows
    full = _call(svt, w, tau, delta, 4, precision="fp64", t=1, dt=2)
    fwd = _call(svt, w, tau, delta, 4, precision="fp64", t=1, dt=2, with_grad=False)
    assert full["info"]["ritz_grown"] > 0 and full["info"]["k_final"] >= 2, full["info"]
    assert fwd["grad_vals"] is None and np.isnan(fwd["grad_tau"])
    assert fwd["loss"] == full["loss"] and np.array_equal(fwd["x_held"], full["x_held"])
    ref = _reference(w, tau, delta, 4)
    _check_against(full, ref, 1e-6, 1e-8)
    # a threshold below every revealed value with the rank capped: the kept set is not certified
    with pytest.raises(RuntimeError, match="r_max"):
        _call(svt, w, 1e-3, delta, 2, precision="fp64", r_max=2, t=2, dt=1)


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function(svt, device):
    """SVTUnrolled returns X^(T) on the held-out entries; the loss is computed in torch and
    its gradient flows through svt_unrolled_backward.  With host or device tensors it must
    reproduce svt_unrolled_grad (the held-out MSE and its gradient) exactly."""
    import torch
    w = workloads.random_lowrank(36, 36, 2, 0.5, seed=7, n_hold=100)
    idx = (lambda a: torch.from_numpy(a).cuda()) if device == "cuda" else (lambda a: a)
    problem = dict(m=w.m, n=w.n, rows=idx(w.rows), cols=idx(w.cols), held_rows=idx(w.held_rows),
                   held_cols=idx(w.held_cols), steps=4,
                   options=dict(checkpoint_every=2, cg_tol=1e-12, precision="fp64", seed=w.seed))
    vals = torch.tensor(w.vals, dtype=torch.float64, device=device, requires_grad=True)
    tau = torch.tensor(2.0 * np.sqrt(w.m * w.n), dtype=torch.float64, requires_grad=True)
    delta = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
    x = svt.SVTUnrolled.apply(vals, tau, delta, problem)
    assert x.device.type == device and x.shape == (w.held_rows.size,)
    held = torch.tensor(w.held_vals, dtype=torch.float64, device=device)
    loss = ((x - held) ** 2).mean()
    (3.0 * loss).backward()
    direct = svt.unrolled_grad(w.m, w.n, w.rows, w.cols, w.vals, w.held_rows, w.held_cols, w.held_vals,
                               float(tau), float(delta), 4, **problem["options"])
    assert np.array_equal(x.detach().cpu().numpy(), direct["x_held"])
    assert abs(loss.item() - direct["loss"]) <= 1e-14 * direct["loss"]
    np.testing.assert_allclose(vals.grad.cpu().numpy(), 3.0 * direct["grad_vals"], rtol=1e-12, atol=1e-18)
    assert abs(tau.grad.item() - 3.0 * direct["grad_tau"]) <= 1e-12 * abs(direct["grad_tau"])
    assert abs(delta.grad.item() - 3.0 * direct["grad_delta"]) <= 1e-12 * abs(direct["grad_delta"])
    # no gradient wanted: the forward keeps no tape and costs only the forward pass
    with torch.no_grad():
        x2 = svt.SVTUnrolled.apply(vals, tau, delta, problem)
    assert torch.equal(x2, x.detach())


# The full-size differentiable workload: 2000 x 2000 rank 20, 10% observed, 40,000 held-out
# entries, tau = 10,000, delta = 12, 20 iterations in binary32 with checkpoints every 5.
# Gradient of the held-out MSE against the binary64 full-SVD reference and against central
# differences (h = 1e-3) of the binary64 forward, both to 1e-4 relative.
def test_unrolled2000_fp32_gradient(svt):
    w = workloads.make("unrolled2000")
    T = 20
    common = dict(checkpoint_every=5, r_max=200)
    g32 = _call(svt, w, w.tau, w.delta, T, precision="mixed", **common)
    g64 = _call(svt, w, w.tau, w.delta, T, precision="fp64", **common)
    ref = _reference(w, w.tau, w.delta, T)
    h = 1e-3

    def loss(v=w.vals, t=w.tau, d=w.delta):
        return svt.unrolled_grad(w.m, w.n, w.rows, w.cols, v, w.held_rows, w.held_cols, w.held_vals,
                                 t, d, T, seed=w.seed, precision="fp64", with_grad=False,
                                 **common)["loss"]
    fd_tau = (loss(t=w.tau + h) - loss(t=w.tau - h)) / (2 * h)
    fd_delta = (loss(d=w.delta + h) - loss(d=w.delta - h)) / (2 * h)
    direction = np.random.default_rng(2).standard_normal(w.vals.shape)
    fd_vals = (loss(v=w.vals + h * direction) - loss(v=w.vals - h * direction)) / (2 * h)
    report = {
        "info32": g32["info"], "info64": g64["info"],
        "x32": _rel(g32["x_held"], ref.x_held), "x64": _rel(g64["x_held"], ref.x_held),
        "gv32": _rel(g32["grad_vals"], ref.grad_vals), "gv64": _rel(g64["grad_vals"], ref.grad_vals),
        "gtau": (g32["grad_tau"], g64["grad_tau"], ref.grad_tau, fd_tau),
        "gdelta": (g32["grad_delta"], g64["grad_delta"], ref.grad_delta, fd_delta),
        "gdir": (float(np.dot(g32["grad_vals"], direction)), float(np.dot(ref.grad_vals, direction)), fd_vals),
    }
    print(report)
    assert g32["info"]["k0"] == ref.k0 and g64["info"]["k0"] == ref.k0
    assert g32["info"]["cg_capped"] == 0 and g64["info"]["cg_capped"] == 0, report
    # binary64 path: the reference to far below the bar
    assert report["x64"] <= 1e-8 and report["gv64"] <= 1e-6, report
    assert _scalar_close(g64["grad_tau"], ref.grad_tau, 1e-6), report
    assert _scalar_close(g64["grad_delta"], ref.grad_delta, 1e-6), report
    # binary32 path against the reference and the central differences
    assert report["x32"] <= 1e-4 and report["gv32"] <= 1e-4, report
    for got, exact in ((g32["grad_tau"], ref.grad_tau), (g32["grad_delta"], ref.grad_delta),
                       (g32["grad_tau"], fd_tau), (g32["grad_delta"], fd_delta),
                       (report["gdir"][0], fd_vals)):
        assert _scalar_close(got, exact, 1e-4), report


def test_unrolled2000_through_autograd_on_the_device(svt):
    """The 2000 x 2000 workload in binary32 through SVTUnrolled with CUDA tensors: the
    gradient equals svt_unrolled_grad's (the loss's gradient on X^(T) is formed in torch
    instead of in the library, so agreement is to rounding), and a forward-only call
    (no tape) takes the forward time, well under forward + backward."""
    import time
    import torch
    w = workloads.make("unrolled2000")
    d = lambda a: torch.from_numpy(a).cuda()
    problem = dict(m=w.m, n=w.n, rows=d(w.rows), cols=d(w.cols), held_rows=d(w.held_rows),
                   held_cols=d(w.held_cols), steps=20,
                   options=dict(checkpoint_every=5, r_max=200, precision="mixed", seed=w.seed))
    vals = torch.tensor(w.vals, dtype=torch.float32, device="cuda", requires_grad=True)
    held = d(w.held_vals)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x = svt.SVTUnrolled.apply(vals, w.tau, w.delta, problem)
    loss = ((x - held) ** 2).mean()
    loss.backward()
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    t0 = time.perf_counter()
    with torch.no_grad():
        x_fwd = svt.SVTUnrolled.apply(vals, w.tau, w.delta, problem)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    direct = _call(svt, w, w.tau, w.delta, 20, precision="mixed", checkpoint_every=5, r_max=200)
    print(f"\nunrolled2000 through autograd: forward + backward {t_full:.3f} s, forward only {t_fwd:.3f} s")
    assert torch.equal(x_fwd, x.detach())
    assert _rel(x.detach().cpu().numpy(), direct["x_held"]) == 0.0
    assert _rel(vals.grad.double().cpu().numpy(), direct["grad_vals"]) < 1e-6
    assert t_fwd < 0.75 * t_full
