"""GB300 (sm_103a) fast singular value thresholding with R4SVD.

Thin Python binding of the C ABI in ``include/svt_gb300.h``: it marshals torch
tensors (device memory, the current CUDA stream) or numpy arrays (host memory) into
the library calls; every step of the computation runs in the library's CUDA kernels.
There is no CPU fallback: without a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib as L

__all__ = ["SVTError", "options", "Pattern", "gaussian_block", "spmm", "spmm_noalloc", "sampled_update",
           "workspace_size", "r4svd_workspace_size",
           "sampled_update_recycle",
           "r4svd", "complete", "library", "launch_count", "profile_enable", "profile_reset", "profile_read",
           "unrolled_grad", "unrolled_params", "SVTUnrolled", "FP64", "MIXED_FP32"]

FP64 = L.SVT_FP64
MIXED_FP32 = L.SVT_MIXED_FP32
_PREC = {"fp64": FP64, "float64": FP64, "mixed": MIXED_FP32, "fp32": MIXED_FP32,
         "mixed_fp32": MIXED_FP32, FP64: FP64, MIXED_FP32: MIXED_FP32}


class SVTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"svt status {status}: {message}")
        self.status = status


def library():
    return L.load()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the SVT library needs a CUDA device (no CPU fallback exists)")
    return torch


def _check(st):
    if st < 0:
        lib = library()
        raise SVTError(st, lib.svt_last_error().decode())
    return st


def _prec(p):
    try:
        return _PREC[p]
    except KeyError:
        raise ValueError(f"unknown precision {p!r}") from None


def _vdtype(prec):
    torch = _torch()
    return torch.float64 if prec == FP64 else torch.float32


def _stream_ptr():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


RECYCLE = {"all": 0, "kept": 1, "none": 2}
STOP = {"residual": 0, "mae": 1}


def options(precision="fp64", **kw) -> L.Options:
    """svt_options with the library defaults, then the given fields.  recycle may be
    "all" (Algorithm 3), "kept" or "none" (Algorithm 2 every call; with t = r_max the
    fixed-rank randomized SVD)."""
    lib = library()
    o = L.Options()
    lib.svt_default_options(C.byref(o))
    o.precision = _prec(precision)
    for key, val in kw.items():
        if key == "t" and val is None:
            continue
        if key == "recycle" and isinstance(val, str):
            if val not in RECYCLE:
                raise ValueError(f"recycle must be one of {sorted(RECYCLE)}")
            val = RECYCLE[val]
        if key == "stop" and isinstance(val, str):
            if val not in STOP:
                raise ValueError(f"stop must be one of {sorted(STOP)}")
            val = STOP[val]
        if not hasattr(o, key):
            raise TypeError(f"unknown option {key}")
        setattr(o, key, val)
    return o


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _cuda_i32(x):
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32))
    return x.to(device="cuda", dtype=torch.int32).contiguous()


class Pattern:
    """The observed set Lambda sorted into CSR and CSC order on the device."""

    def __init__(self, m, n, rows, cols):
        torch = _torch()
        lib = library()
        self.m, self.n = int(m), int(n)
        r = _cuda_i32(rows)
        c = _cuda_i32(cols)
        h = C.c_void_p()
        _check(lib.svt_pattern_create(self.m, self.n, r.numel(), _ptr(r), _ptr(c), _stream_ptr(),
                                      C.byref(h)))
        self._h = h
        self.nnz = int(lib.svt_pattern_nnz(h))
        self._torch = torch

    @property
    def handle(self):
        return self._h

    def export(self):
        torch = self._torch
        dev = dict(device="cuda", dtype=torch.int32)
        out = dict(row_ptr=torch.empty(self.m + 1, **dev), col_idx=torch.empty(self.nnz, **dev),
                   csr_src=torch.empty(self.nnz, **dev), col_ptr=torch.empty(self.n + 1, **dev),
                   row_idx=torch.empty(self.nnz, **dev), perm=torch.empty(self.nnz, **dev))
        _check(library().svt_pattern_export(self._h, *[_ptr(out[k]) for k in
                                            ("row_ptr", "col_idx", "csr_src", "col_ptr", "row_idx",
                                             "perm")], _stream_ptr()))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            library().svt_pattern_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gaussian_block(seed, it, block, n, w):
    torch = _torch()
    out = torch.empty((n, w), device="cuda", dtype=torch.float64)
    _check(library().svt_gaussian_block(int(seed), int(it) & 0xFFFFFFFF, int(block) & 0xFFFFFFFF, n, w,
                                        _ptr(out), max(w, 1), _stream_ptr()))
    return out


def _check_spmm_operands(pattern, y, W, transpose):
    """The C entry points cannot see buffer sizes: a short y or W would make the kernels
    read past its end, so the sizes are checked here, before any work is queued."""
    if y.dim() != 1 or y.numel() != pattern.nnz:
        raise ValueError(f"y_csr must hold the pattern's {pattern.nnz} values, got shape {tuple(y.shape)}")
    rows_in = pattern.m if transpose else pattern.n
    if W.dim() != 2 or W.shape[0] != rows_in:
        raise ValueError(f"W must have {rows_in} rows ({'m' if transpose else 'n'}), got shape "
                         f"{tuple(W.shape)}")


def spmm(pattern: Pattern, y_csr, W, transpose=False, precision="fp64"):
    """Y W (transpose False, W n x w) or Y^T W (transpose True, W m x w)."""
    torch = _torch()
    prec = _prec(precision)
    dt = _vdtype(prec)
    y = y_csr.to(device="cuda", dtype=dt).contiguous()
    W = W.to(device="cuda", dtype=dt).contiguous()
    _check_spmm_operands(pattern, y, W, transpose)
    w = W.shape[1]
    rows = pattern.n if transpose else pattern.m
    out = torch.empty((rows, w), device="cuda", dtype=dt)
    _check(library().svt_spmm(pattern.handle, prec, 1 if transpose else 0, _ptr(y), _ptr(W), max(w, 1),
                              w, _ptr(out), max(w, 1), _stream_ptr()))
    return out


def spmm_noalloc(pattern: Pattern, y_csr, W, out, transpose=False, precision="fp64"):
    """Like spmm, but the library allocates nothing: its scratch is a fixed device array
    (see svt_spmm_noalloc in the C header).  The caller supplies `out` (rows x w).  W and
    out are row-major with unit column stride; their leading dimensions are their row
    strides, so either may be the first w columns of a wider array (a leading dimension
    that is a multiple of 4 binary32 or 2 binary64 values lets the rows load as 16-byte
    vectors)."""
    prec = _prec(precision)
    dt = _vdtype(prec)
    assert y_csr.is_cuda and y_csr.dtype == dt and y_csr.is_contiguous()
    assert W.is_cuda and W.dtype == dt and W.dim() == 2 and W.stride(1) == 1
    _check_spmm_operands(pattern, y_csr, W, transpose)
    w = W.shape[1]
    rows = pattern.n if transpose else pattern.m
    assert out.is_cuda and out.dtype == dt and out.dim() == 2 and out.stride(1) == 1
    assert tuple(out.shape) == (rows, w)
    ldw = max(W.stride(0), w, 1) if W.shape[0] > 1 else max(w, 1)
    ldo = max(out.stride(0), w, 1) if out.shape[0] > 1 else max(w, 1)
    _check(library().svt_spmm_noalloc(pattern.handle, prec, 1 if transpose else 0, _ptr(y_csr), _ptr(W),
                                      ldw, w, _ptr(out), ldo, _stream_ptr()))
    return out


def sampled_update(pattern: Pattern, U, W, a_csr, y_csr, delta, precision="fp64"):
    """In place on y_csr: y += delta (a - (U W^T) on Lambda); returns (sum d^2, sum |d|, sum y^2)."""
    prec = _prec(precision)
    dt = _vdtype(prec)
    U = U.to(device="cuda", dtype=dt).contiguous()
    W = W.to(device="cuda", dtype=dt).contiguous()
    a = a_csr.to(device="cuda", dtype=dt).contiguous()
    assert y_csr.is_cuda and y_csr.dtype == dt and y_csr.is_contiguous()
    k = U.shape[1]
    sums = (C.c_double * 3)()
    _check(library().svt_sampled_update(pattern.handle, prec, _ptr(U), max(k, 1), _ptr(W), max(k, 1), k,
                                        _ptr(a), _ptr(y_csr), float(delta), sums, _stream_ptr()))
    return tuple(sums)


def sampled_update_recycle(pattern: Pattern, U, W, a_csc, y_csc, delta, precision="fp64"):
    """In place on y_csc (CSC order): y += delta (a - (U[:, :k] W^T) on Lambda), with k the
    width of W; returns (Bt, sums) with Bt (n x r) = y_new^T U and sums as in
    sampled_update."""
    torch = _torch()
    prec = _prec(precision)
    dt = _vdtype(prec)
    vec = 2 if dt == torch.float64 else 4
    m, r = U.shape
    k = W.shape[1]
    n = W.shape[0]
    ldu, ldw = -(-r // vec) * vec, max(-(-k // vec) * vec, vec)
    Up = torch.zeros((m, ldu), device="cuda", dtype=dt)
    Up[:, :r] = U.to(device="cuda", dtype=dt)
    Wp = torch.zeros((n, ldw), device="cuda", dtype=dt)
    Wp[:, :k] = W.to(device="cuda", dtype=dt)
    a = a_csc.to(device="cuda", dtype=dt).contiguous()
    assert y_csc.is_cuda and y_csc.dtype == dt and y_csc.is_contiguous()
    Bt = torch.empty((n, r), device="cuda", dtype=dt)
    sums = (C.c_double * 3)()
    _check(library().svt_sampled_update_recycle(pattern.handle, prec, _ptr(Up), ldu, r, _ptr(Wp), ldw,
                                                k, _ptr(a), _ptr(y_csc), float(delta), _ptr(Bt), r,
                                                sums, _stream_ptr()))
    return Bt, tuple(sums)


def _ws_args(workspace):
    """(pointer, bytes) of a caller workspace: a CUDA tensor (any dtype, contiguous), or None."""
    if workspace is None:
        return C.c_void_p(0), 0
    assert workspace.is_cuda and workspace.is_contiguous()
    return C.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


def workspace_size(m, n, nnz, n_eval=0, cap=None, precision="fp64", **kw):
    """Device bytes a solve (complete) takes from a caller workspace (svt_workspace_size)."""
    o = options(precision, **kw)
    if cap is None:
        cap = min(m, n, o.r_max) if o.r_max > 0 else min(m, n)
    return int(library().svt_workspace_size(m, n, nnz, n_eval, cap, C.byref(o)))


def r4svd_workspace_size(m, n, nnz, precision="fp64", **kw):
    """Device bytes an r4svd call takes from a caller workspace."""
    o = options(precision, **kw)
    return int(library().svt_r4svd_workspace_size(m, n, nnz, C.byref(o)))


def r4svd(pattern: Pattern, y_csr, eps_thr, it, U_prev=None, precision="fp64", workspace=None, **kw):
    """One R4SVD call (Algorithm 3; Algorithm 2 when U_prev is None).  workspace: a CUDA
    tensor of at least r4svd_workspace_size bytes, from which the call takes its scratch
    instead of allocating."""
    torch = _torch()
    o = options(precision, **kw)
    o.stream = _stream_ptr().value
    dt = _vdtype(o.precision)
    m, n = pattern.m, pattern.n
    r_cap = min(m, n, o.r_max) if o.r_max > 0 else min(m, n)
    y = y_csr.to(device="cuda", dtype=dt).contiguous()
    s = 0 if U_prev is None else int(U_prev.shape[1])
    Up = None if U_prev is None else U_prev.to(device="cuda", dtype=dt).contiguous()
    U = torch.zeros((m, r_cap), device="cuda", dtype=dt)
    V = torch.zeros((n, r_cap), device="cuda", dtype=dt)
    S = torch.zeros(r_cap, device="cuda", dtype=torch.float64)
    r, eps, blocks = C.c_int32(0), C.c_double(0), C.c_int32(0)
    _check(library().svt_r4svd(pattern.handle, _ptr(y), _ptr(Up), max(s, 1), s, float(eps_thr),
                               int(it) & 0xFFFFFFFF, C.byref(o), _ptr(U), r_cap, _ptr(S), _ptr(V), r_cap,
                               C.byref(r), C.byref(eps), C.byref(blocks), *_ws_args(workspace)))
    rr = r.value
    return dict(U=U[:, :rr], S=S[:rr], V=V[:, :rr], r=rr, eps=eps.value, blocks=blocks.value)


@dataclass
class Completion:
    U: object
    S: object
    V: object
    k: int
    iters: int
    status: int
    rel_residual: float
    mae: float
    k0: int
    spec_norm: float
    r: int
    seconds_pattern: float
    seconds_total: float
    log: list

    @property
    def converged(self):
        return self.status == L.SVT_OK


def profile_enable(on=True):
    library().svt_profile_enable(1 if on else 0)


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(library().svt_launch_count())


def profile_reset():
    library().svt_profile_reset()


def profile_read(cap=64):
    """Per-kernel-class totals: name -> dict(launches, ms, bytes)."""
    names = C.create_string_buffer(32 * cap)
    launches = (C.c_int64 * cap)()
    ms = (C.c_double * cap)()
    nbytes = (C.c_double * cap)()
    count = library().svt_profile_read(cap, names, launches, ms, nbytes)
    out = {}
    for i in range(min(count, cap)):
        nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = dict(launches=int(launches[i]), ms=float(ms[i]), bytes=float(nbytes[i]))
    return out


def _log_list(buf, n):
    keys = [f[0] for f in L.IterLog._fields_]
    return [{k: getattr(buf[i], k) for k in keys} for i in range(n)]


def complete(m, n, rows, cols, vals, tau, delta, tol, maxit, precision="fp64", log=True,
             on_host=None, eval_set=None, workspace=None, **kw) -> Completion:
    """Algorithm 4 on (rows, cols, vals).

    Host inputs (numpy) are copied to the device inside the call and the factors come
    back as numpy arrays; device inputs (torch CUDA tensors) give device outputs.
    eval_set = (rows, cols, vals) of held-out entries adds their MAE after every
    iteration to the log ("mae_eval"); stop="mae" ends on the training MAE instead of the
    relative residual.  workspace: a CUDA tensor of at least workspace_size(...) bytes from
    which the solve takes every device array instead of allocating.
    """
    torch = _torch()
    o = options(precision, **kw)
    o.stream = _stream_ptr().value
    dt = _vdtype(o.precision)
    r_cap = min(m, n, o.r_max) if o.r_max > 0 else min(m, n)
    host = isinstance(vals, np.ndarray) if on_host is None else on_host
    if host and not isinstance(vals, np.ndarray):
        # torch CPU tensors (e.g. pinned): pass their host pointers straight through
        want = torch.float64 if o.precision == FP64 else torch.float32
        assert rows.dtype == torch.int32 and cols.dtype == torch.int32 and vals.dtype == want
        assert not (rows.is_cuda or cols.is_cuda or vals.is_cuda)
        U = torch.zeros((m, r_cap), dtype=torch.float64).pin_memory()
        S = torch.zeros(r_cap, dtype=torch.float64).pin_memory()
        V = torch.zeros((n, r_cap), dtype=torch.float64).pin_memory()
        args = [_ptr(rows.contiguous()), _ptr(cols.contiguous()), _ptr(vals.contiguous())]
        outs = [_ptr(U), _ptr(S), _ptr(V)]
        nnz = rows.numel()
        keep = (rows, cols, vals)
    elif host:
        np_dt = np.float64 if o.precision == FP64 else np.float32
        rows_h = np.ascontiguousarray(rows, dtype=np.int32)
        cols_h = np.ascontiguousarray(cols, dtype=np.int32)
        vals_h = np.ascontiguousarray(vals, dtype=np_dt)
        U = np.zeros((m, r_cap)); S = np.zeros(r_cap); V = np.zeros((n, r_cap))
        args = [rows_h.ctypes.data_as(C.c_void_p), cols_h.ctypes.data_as(C.c_void_p),
                vals_h.ctypes.data_as(C.c_void_p)]
        outs = [U.ctypes.data_as(C.c_void_p), S.ctypes.data_as(C.c_void_p), V.ctypes.data_as(C.c_void_p)]
        nnz = rows_h.shape[0]
        keep = (rows_h, cols_h, vals_h)
    else:
        rows_d, cols_d = _cuda_i32(rows), _cuda_i32(cols)
        vals_d = vals.to(device="cuda", dtype=dt).contiguous()
        U = torch.zeros((m, r_cap), device="cuda", dtype=torch.float64)
        S = torch.zeros(r_cap, device="cuda", dtype=torch.float64)
        V = torch.zeros((n, r_cap), device="cuda", dtype=torch.float64)
        args = [_ptr(rows_d), _ptr(cols_d), _ptr(vals_d)]
        outs = [_ptr(U), _ptr(S), _ptr(V)]
        nnz = rows_d.numel()
        keep = (rows_d, cols_d, vals_d)
    res = L.Result()
    log_cap = maxit if log else 0
    logbuf = (L.IterLog * max(log_cap, 1))()
    eval_args, n_eval, keep_eval = [C.c_void_p(0)] * 3, 0, None
    if eval_set is not None:
        er, ec, ev = eval_set
        np_dt = np.float64 if o.precision == FP64 else np.float32
        keep_eval = (np.ascontiguousarray(np.asarray(er), dtype=np.int32),
                     np.ascontiguousarray(np.asarray(ec), dtype=np.int32),
                     np.ascontiguousarray(np.asarray(ev), dtype=np_dt))
        eval_args = [a.ctypes.data_as(C.c_void_p) for a in keep_eval]
        n_eval = keep_eval[0].shape[0]
    st = library().svt_complete_eval(m, n, nnz, *args, n_eval, *eval_args, float(tau), float(delta),
                                     float(tol), int(maxit), C.byref(o), *outs, r_cap, C.byref(res),
                                     logbuf, log_cap, *_ws_args(workspace))
    del keep, keep_eval
    _check(st)
    k = res.k
    return Completion(U=U[:, :k], S=S[:k], V=V[:, :k], k=k, iters=res.iters, status=res.status,
                      rel_residual=res.rel_residual, mae=res.mae, k0=res.k0, spec_norm=res.spec_norm,
                      r=res.r, seconds_pattern=res.seconds_pattern, seconds_total=res.seconds_total,
                      log=_log_list(logbuf, res.log_len))


def unrolled_params(precision="fp64", **kw):
    """svt_unrolled_params with the library defaults for `precision`, then `kw` applied."""
    up = L.UnrolledParams()
    library().svt_unrolled_default_params(C.byref(up), _prec(precision))
    names = {f[0] for f in L.UnrolledParams._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown unrolled parameter {k!r}")
        setattr(up, k, v)
    return up


_UNROLLED_KEYS = ("checkpoint_every", "cg_maxit", "ritz_maxit", "cg_tol", "ritz_tol")


def unrolled_grad(m, n, rows, cols, vals, held_rows, held_cols, held_vals, tau, delta, steps,
                  precision="fp64", with_grad=True, **kw):
    """Unrolled SVT and its gradient (svt_unrolled_grad): returns a dict with the held-out
    MSE `loss`, `grad_vals` (numpy, input order), `grad_tau`, `grad_delta`, `x_held` and
    the solver info.  Index and value arrays are host (numpy) arrays.  Keywords named like
    the fields of svt_unrolled_params (checkpoint_every, cg_tol, cg_maxit, ritz_tol,
    ritz_maxit) set those; the rest go to the solver options.  with_grad=False runs the
    forward only (grad_vals None, grad_tau and grad_delta NaN)."""
    _torch()
    up = unrolled_params(precision, steps=int(steps),
                         **{k: kw.pop(k) for k in list(kw) if k in _UNROLLED_KEYS})
    o = options(precision, **kw)
    o.stream = _stream_ptr().value
    np_dt = np.float64 if o.precision == FP64 else np.float32
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np_dt)
    hr = np.ascontiguousarray(held_rows, dtype=np.int32)
    hc = np.ascontiguousarray(held_cols, dtype=np.int32)
    hv = np.ascontiguousarray(held_vals, dtype=np_dt)
    grad = np.zeros(r.shape[0])
    xh = np.zeros(hr.shape[0])
    out3 = np.zeros(3)
    info = L.UnrolledInfo()
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(library().svt_unrolled_grad(m, n, r.shape[0], p(r), p(c), p(v), hr.shape[0], p(hr), p(hc),
                                       p(hv), float(tau), float(delta), C.byref(up), C.byref(o),
                                       p(grad) if with_grad else None, p(xh), p(out3), C.byref(info)))
    keys = [f[0] for f in L.UnrolledInfo._fields_]
    return dict(loss=float(out3[0]), grad_vals=grad if with_grad else None, grad_tau=float(out3[1]),
                grad_delta=float(out3[2]),
                x_held=xh, info={k: getattr(info, k) for k in keys})


class _Tape:
    """Owner of a C-side unrolled tape (released when the Python object goes away)."""

    def __init__(self, handle, nnz, nheld):
        self.handle, self.nnz, self.nheld = handle, nnz, nheld

    def release(self):
        if self.handle is not None and self.handle.value:
            library().svt_unrolled_tape_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def _host_or_device_ptr(x, dtype):
    """(pointer, keep-alive) of a numpy array or torch tensor with the given numpy dtype."""
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=dtype)
        return a.ctypes.data_as(C.c_void_p), a
    t = x.detach().contiguous()
    return C.c_void_p(t.data_ptr()), t


def _make_unrolled_function():
    torch = _torch()

    class SVTUnrolled(torch.autograd.Function):
        """X^(T) of unrolled SVT on the held-out entries, as a differentiable function of the
        observed values, tau and delta.  forward runs svt_unrolled_forward on the device
        (vals may be a CUDA tensor; nothing is copied through the host) and keeps the
        checkpoint tape only when a gradient may be needed; backward hands the incoming
        gradient on the predictions to svt_unrolled_backward, which replays the tape.
        problem: m, n, rows, cols, held_rows, held_cols (numpy or CUDA int32), steps and
        options (keywords of unrolled_grad)."""

        @staticmethod
        def forward(ctx, vals, tau, delta, problem):
            opts = dict(problem.get("options", {}))
            prec = opts.get("precision", "fp64")
            up = unrolled_params(prec, steps=int(problem["steps"]),
                                 **{k: opts.pop(k) for k in list(opts) if k in _UNROLLED_KEYS})
            o = options(**opts)
            o.stream = _stream_ptr().value
            want = torch.float64 if o.precision == FP64 else torch.float32
            v = vals.detach().to(want).contiguous()
            r, kr = _host_or_device_ptr(problem["rows"], np.int32)
            c, kc = _host_or_device_ptr(problem["cols"], np.int32)
            hr, khr = _host_or_device_ptr(problem["held_rows"], np.int32)
            hc, khc = _host_or_device_ptr(problem["held_cols"], np.int32)
            nnz, nh = v.numel(), int(khr.shape[0])
            x = torch.empty(nh, dtype=torch.float64, device=vals.device)
            need = any(ctx.needs_input_grad[:3])
            h = C.c_void_p()
            info = L.UnrolledInfo()
            _check(library().svt_unrolled_forward(problem["m"], problem["n"], nnz, r, c, C.c_void_p(v.data_ptr()),
                                                  nh, hr, hc, float(tau), float(delta), C.byref(up),
                                                  C.byref(o), C.c_void_p(x.data_ptr()), C.byref(info),
                                                  C.byref(h) if need else None))
            del kr, kc, khr, khc
            ctx.tape = _Tape(h, nnz, nh) if need else None
            ctx.info = {f[0]: getattr(info, f[0]) for f in L.UnrolledInfo._fields_}
            ctx.vals_meta = (vals.dtype, vals.device)
            ctx.scalar_meta = [(t.dtype, t.device) if torch.is_tensor(t) else None for t in (tau, delta)]
            return x

        @staticmethod
        def backward(ctx, g):
            tape = ctx.tape
            if tape is None:
                return None, None, None, None
            dtype, device = ctx.vals_meta
            gx = g.detach().to(device=device, dtype=torch.float64).contiguous()
            grad = torch.empty(tape.nnz, dtype=torch.float64, device=device)
            gtd = torch.empty(2, dtype=torch.float64, device=device)
            info = L.UnrolledInfo()
            try:
                _check(library().svt_unrolled_backward(tape.handle, C.c_void_p(gx.data_ptr()),
                                                       C.c_void_p(grad.data_ptr()), C.c_void_p(gtd.data_ptr()),
                                                       C.byref(info)))
            finally:
                tape.release()
            ctx.info = {f[0]: getattr(info, f[0]) for f in L.UnrolledInfo._fields_}
            gs = [None if meta is None else gtd[i].to(dtype=meta[0], device=meta[1])
                  for i, meta in enumerate(ctx.scalar_meta)]
            return grad.to(dtype), gs[0], gs[1], None

    return SVTUnrolled


class _LazyUnrolled:
    _fn = None

    def apply(self, *args):
        if _LazyUnrolled._fn is None:
            _LazyUnrolled._fn = _make_unrolled_function()
        return _LazyUnrolled._fn.apply(*args)


SVTUnrolled = _LazyUnrolled()
