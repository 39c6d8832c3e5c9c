"""Thin ctypes binding of the C ABI in include/uoi.h (argument marshalling only).

Every function here forwards pointers and sizes to libuoi_gb300.so; all the
arithmetic runs in the CUDA kernels.  Arrays may be numpy arrays (host memory)
or torch CUDA tensors (device memory); outputs are returned in the same kind as
the main input.  Importing this module raises if the library is missing: there
is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, OK_WITH_WARNINGS = 0, 1
ERR_INVALID_ARG, ERR_NONFINITE, ERR_NOT_PD, ERR_CUDA = -1, -2, -3, -4
ERR_OOM, ERR_TIMEOUT, ERR_BOUNDS, ERR_UNSUPPORTED = -5, -6, -7, -8
BAG_MEDIAN, BAG_MEAN = 0, 1
SPLIT_PER_BOOTSTRAP, SPLIT_FIXED = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
WARM_NONE, WARM_PATH, WARM_LEARNED = 0, 1, 2


class UoiParams(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("B1", C.c_int32), ("B2", C.c_int32), ("q", C.c_int32),
        ("lambdas", C.c_void_p), ("lambda_min_ratio", C.c_double), ("rho", C.c_double),
        ("abs_tol", C.c_double), ("rel_tol", C.c_double), ("max_iter", C.c_int32),
        ("train_frac", C.c_double), ("seed", C.c_uint64), ("problem_id", C.c_uint64),
        ("block_len", C.c_int64), ("bagging", C.c_int32), ("split_mode", C.c_int32),
        ("precision", C.c_int32), ("warm_start", C.c_int32), ("mlp_weights_path", C.c_char_p),
        ("stream", C.c_void_p), ("intercept", C.c_int32), ("block_mode", C.c_int32),
    ]


class UoiDiag(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("ms_total", C.c_float), ("ms_bootstrap", C.c_float),
        ("ms_gram", C.c_float), ("ms_factor", C.c_float), ("ms_admm", C.c_float),
        ("ms_support", C.c_float), ("ms_estimation", C.c_float),
        ("admm_columns", C.c_int64), ("admm_nonconverged", C.c_int64),
        ("admm_iterations", C.c_int64), ("admm_max_iterations", C.c_int32),
        ("ols_singular", C.c_int64), ("gpu_launches", C.c_int64),
        ("ms_gram_tc", C.c_float), ("n_gram_tc", C.c_int64), ("flops_gram_tc", C.c_double),
        ("ms_xupdate", C.c_float), ("n_xupdate", C.c_int64), ("flops_xupdate", C.c_double),
        ("bytes_xupdate", C.c_double), ("warm_start_used", C.c_int32),
        ("ols_fp64", C.c_int64), ("admm_near_threshold", C.c_int64),
        ("admm_iter_hist", C.c_int64 * 8),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            if name == "struct_size":
                continue
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, C.Array) else v
        return out


class UoiTrace(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "lambdas", "sel_weights", "est_weights", "est_eval", "sel_beta", "sel_iters", "sel_conv",
        "family", "est_loss", "est_jstar", "est_beta", "est_singular")]


_lib = None
_checked = None


def lib():
    """Load (building if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libuoi_gb300.so is missing; the CUDA path cannot run")
        _lib = _configure(C.CDLL(path))
    return _lib


def checked_lib():
    """Load (building if needed) the checked build (UOI_BOUNDS_CHECK=1), a separate
    library with the same entry points; use it through use_library."""
    global _checked
    if _checked is None:
        path = _build.build(checked=True)
        if not os.path.exists(path):
            raise RuntimeError("libuoi_gb300_checked.so is missing")
        _checked = _configure(C.CDLL(path))
    return _checked


class use_library:
    """with use_library(L): the wrappers of this module call library L."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _lib
        lib()
        self.prev, _lib = _lib, self.L
        return self.L

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev


def _configure(L):
    if True:
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.uoi_params_default.argtypes = [C.POINTER(UoiParams)]
        L.uoi_lasso_fit.argtypes = [vp, vp, i64, i64, C.POINTER(UoiParams), vp, vp, C.POINTER(UoiDiag)]
        L.uoi_var_fit.argtypes = [vp, i64, i64, i32, C.POINTER(UoiParams), vp, vp, C.POINTER(UoiDiag)]
        L.uoi_lasso_fit_batch.argtypes = [i32, vp, vp, vp, vp, C.POINTER(UoiParams), vp, vp, vp, i32]
        L.uoi_fit_traced.argtypes = [vp, i64, vp, i64, i64, i64, i64, C.POINTER(UoiParams), vp,
                                     C.POINTER(UoiTrace), C.POINTER(UoiDiag)]
        L.lasso_admm_batch.argtypes = [vp, vp, i64, i64, i64, vp, i32, vp, i32, d, d, d, i32, i32,
                                       i32, vp, vp, vp, vp]
        L.uoi_weighted_moments.argtypes = [vp, vp, i64, i64, i64, vp, i32, i32, vp, vp, vp]
        L.lasso_admm_batch_noalloc.argtypes = [vp, vp, i64, i64, i64, vp, i32, vp, i32, d, d, d,
                                               i32, i32, vp, vp, vp, vp]
        L.uoi_ws_param_count.restype = i64
        L.uoi_ws_create.argtypes = [C.c_uint64, C.POINTER(vp)]
        L.uoi_ws_load.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.uoi_ws_save.argtypes = [vp, C.c_char_p]
        L.uoi_ws_free.argtypes = [vp]
        L.uoi_ws_set_params.argtypes = [vp, vp]
        L.uoi_ws_get_params.argtypes = [vp, vp]
        L.uoi_ws_forward.argtypes = [vp, vp, i64, vp]
        L.uoi_ws_loss_grad.argtypes = [vp, vp, vp, i64, C.POINTER(d), vp]
        L.uoi_ws_train.argtypes = [vp, vp, vp, i64, i32, i32, C.c_float, C.c_uint64, C.POINTER(d)]
        L.uoi_ws_dataset.argtypes = [vp, vp, i64, i64, i64, vp, i32, vp, i32, d, d, d, i32, vp, vp, vp]
        L.uoi_selftest_wait.argtypes = [C.c_uint64, i32, C.POINTER(d), vp]
        L.uoi_selftest_index_check.argtypes = [i64, i64, vp]
        L.uoi_status_string.argtypes = [C.c_int]
        L.uoi_status_string.restype = C.c_char_p
        L.uoi_get_last_error_detail.argtypes = [C.c_char_p, C.c_size_t]
        L.uoi_shutdown.argtypes = []
    return L


EXPORTED = ("uoi_params_default", "uoi_lasso_fit", "uoi_lasso_fit_batch", "uoi_var_fit", "uoi_fit_traced",
            "lasso_admm_batch", "lasso_admm_batch_noalloc", "uoi_weighted_moments",
            "uoi_ws_param_count", "uoi_ws_create", "uoi_ws_load", "uoi_ws_save", "uoi_ws_free",
            "uoi_ws_set_params", "uoi_ws_get_params", "uoi_ws_forward", "uoi_ws_loss_grad",
            "uoi_ws_train", "uoi_ws_dataset", "uoi_selftest_wait", "uoi_selftest_index_check", "uoi_status_string", "uoi_get_last_error_detail",
            "uoi_shutdown")


class UoiError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__(f"status {status}: {detail}")
        self.status = status


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().uoi_get_last_error_detail(buf, 1024)
    return buf.value.decode()


def _check(st):
    if st < 0:
        raise UoiError(st, last_error())
    return st


# ----------------------------------------------------------------------------
# array helpers: numpy (host) or torch CUDA tensors (device)
# ----------------------------------------------------------------------------
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _prep(a, dtype):
    if _is_torch(a):
        import torch
        tmap = {np.float64: torch.float64, np.uint32: torch.int32, np.uint8: torch.uint8}
        t = a.contiguous()
        if dtype is np.uint32:
            return t.to(torch.int32) if t.dtype != torch.int32 else t
        return t.to(tmap[dtype])
    return np.ascontiguousarray(a, dtype=dtype)


def _empty(like, shape, dtype):
    if _is_torch(like):
        import torch
        tmap = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
                np.uint32: torch.int32, np.uint64: torch.int64}
        return torch.empty(shape, dtype=tmap[dtype], device=like.device)
    return np.empty(shape, dtype=dtype)


def make_params(B1=20, B2=20, q=16, lambdas=None, lambda_min_ratio=1e-3, rho=1.0, abs_tol=1e-6,
                rel_tol=1e-6, max_iter=1000, train_frac=0.8, seed=0, problem_id=0, block_len=0,
                bagging=BAG_MEDIAN, split_mode=SPLIT_PER_BOOTSTRAP, precision=PREC_FP64,
                warm_start=WARM_PATH, stream=None, mlp_weights_path=None, intercept=0, block_mode=0):
    prm = UoiParams()
    lib().uoi_params_default(C.byref(prm))
    prm.B1, prm.B2, prm.q = B1, B2, q
    keep = None
    if lambdas is not None:
        keep = _prep(lambdas, np.float64)
        prm.lambdas = _ptr(keep)
    prm.lambda_min_ratio = lambda_min_ratio
    prm.rho, prm.abs_tol, prm.rel_tol, prm.max_iter = rho, abs_tol, rel_tol, max_iter
    prm.train_frac, prm.seed, prm.problem_id = train_frac, seed, problem_id
    prm.block_len, prm.bagging, prm.split_mode = block_len, bagging, split_mode
    prm.precision, prm.warm_start = precision, warm_start
    prm.stream = stream
    prm.intercept = int(intercept)
    prm.block_mode = int(block_mode)
    if mlp_weights_path:
        prm.mlp_weights_path = mlp_weights_path.encode()
    return prm, keep


def uoi_fit_traced(X, Y, trace=True, **kw):
    """General fit of Y (m x r) on X (m x p); returns dict(beta, status, diag, trace...).
    beta and est_beta hold p + 1 values per response with intercept=1 (mu last)."""
    X = _prep(X, np.float64)
    Y = _prep(Y, np.float64)
    if Y.ndim == 1:
        Y = Y.reshape(-1, 1)
    m, p = X.shape
    r = Y.shape[1]
    prm, keep = make_params(**kw)
    B1, B2, q = prm.B1, prm.B2, prm.q
    W = (p + 63) // 64
    pe = p + (1 if prm.intercept else 0)
    beta = _empty(X, (r, pe), np.float64)
    out = {}
    tr = None
    if trace:
        shapes = dict(lambdas=((q,), np.float64), sel_weights=((B1, m), np.uint32),
                      est_weights=((B2, m), np.uint32), est_eval=((B2, m), np.uint8),
                      sel_beta=((B1, q, r, p), np.float64), sel_iters=((B1, q, r), np.int32),
                      sel_conv=((B1, q, r), np.uint8), family=((q, r, W), np.uint64),
                      est_loss=((B2, q, r), np.float64), est_jstar=((B2,), np.int32),
                      est_beta=((B2, r, pe), np.float64), est_singular=((B2, q, r), np.int32))
        tr = UoiTrace()
        for name, (shape, dt) in shapes.items():
            out[name] = _empty(X, shape, dt)
            setattr(tr, name, _ptr(out[name]))
    diag = UoiDiag()
    diag.struct_size = C.sizeof(UoiDiag)
    st = lib().uoi_fit_traced(_ptr(X), p, _ptr(Y), r, m, p, r, C.byref(prm), _ptr(beta),
                              C.byref(tr) if tr is not None else None, C.byref(diag))
    del keep
    _check(st)
    out.update(beta=beta, status=st, diag=diag.as_dict())
    return out


def uoi_lasso_fit_batch(Xs, ys, streams=0, **kw):
    """Independent UoI_LASSO problems (uneven n, p) in one call; returns a list of
    dicts (beta, status, diag) in input order.  Problem i uses problem_id + i."""
    count = len(Xs)
    Xs = [_prep(X, np.float64) for X in Xs]
    ys = [_prep(y, np.float64) for y in ys]
    prm, keep = make_params(**kw)
    betas = [_empty(X, (X.shape[1],), np.float64) for X in Xs]
    xa = (C.c_void_p * count)(*[_ptr(X) for X in Xs])
    ya = (C.c_void_p * count)(*[_ptr(y) for y in ys])
    na = (C.c_int64 * count)(*[X.shape[0] for X in Xs])
    pa = (C.c_int64 * count)(*[X.shape[1] for X in Xs])
    ba = (C.c_void_p * count)(*[_ptr(b) for b in betas])
    sta = (C.c_int32 * count)()
    diags = (UoiDiag * count)()
    for dg in diags:
        dg.struct_size = C.sizeof(UoiDiag)
    st = lib().uoi_lasso_fit_batch(count, C.cast(xa, C.c_void_p), C.cast(ya, C.c_void_p),
                                   C.cast(na, C.c_void_p), C.cast(pa, C.c_void_p), C.byref(prm),
                                   C.cast(ba, C.c_void_p), C.cast(sta, C.c_void_p),
                                   C.cast(diags, C.c_void_p), streams)
    del keep
    _check(st)
    return [dict(beta=betas[i], status=int(sta[i]), diag=diags[i].as_dict()) for i in range(count)]


def uoi_lasso_fit(X, y, family=False, **kw):
    X = _prep(X, np.float64)
    y = _prep(y, np.float64)
    n, p = X.shape
    prm, keep = make_params(**kw)
    beta = _empty(X, (p,), np.float64)
    fam = _empty(X, (prm.q, (p + 63) // 64), np.uint64) if family else None
    diag = UoiDiag()
    diag.struct_size = C.sizeof(UoiDiag)
    st = lib().uoi_lasso_fit(_ptr(X), _ptr(y), n, p, C.byref(prm), _ptr(beta), _ptr(fam),
                             C.byref(diag))
    del keep
    _check(st)
    return dict(beta=beta, family=fam, status=st, diag=diag.as_dict())


def uoi_var_fit(series, order=1, **kw):
    S = _prep(series, np.float64)
    N, p = S.shape
    prm, keep = make_params(**kw)
    A = _empty(S, (max(int(order), 1), p, p), np.float64)
    mu = _empty(S, (p,), np.float64)
    diag = UoiDiag()
    diag.struct_size = C.sizeof(UoiDiag)
    st = lib().uoi_var_fit(_ptr(S), N, p, order, C.byref(prm), _ptr(A), _ptr(mu), C.byref(diag))
    del keep
    _check(st)
    return dict(A=A, mu=mu, status=st, diag=diag.as_dict())


def lasso_admm_batch(X, Y, weights, lambdas, rho=1.0, abs_tol=1e-6, rel_tol=1e-6, max_iter=1000,
                     precision=PREC_FP64, warm_start=WARM_PATH, stream=None):
    X = _prep(X, np.float64)
    Y = _prep(Y, np.float64)
    if Y.ndim == 1:
        Y = Y.reshape(-1, 1)
    n, p = X.shape
    r = Y.shape[1]
    lam = _prep(lambdas, np.float64)
    q = lam.shape[0]
    if weights is None:
        B, w = 1, None
    else:
        w = _prep(weights, np.uint32)
        w = w.reshape(-1, n)
        B = w.shape[0]
    beta = _empty(X, (B, q, r, p), np.float64)
    iters = _empty(X, (B, q, r), np.int32)
    conv = _empty(X, (B, q, r), np.uint8)
    st = lib().lasso_admm_batch(_ptr(X), _ptr(Y), n, p, r, _ptr(w), B, _ptr(lam), q, rho, abs_tol,
                                rel_tol, max_iter, precision, warm_start, _ptr(beta), _ptr(iters),
                                _ptr(conv), stream)
    _check(st)
    return dict(beta=beta, iters=iters, conv=conv, status=st)


def weighted_moments(X, Y, weights, precision=PREC_FP64, stream=None):
    """G_k = X^T diag(w_k) X and B_k = X^T diag(w_k) Y for each weight row k."""
    X = _prep(X, np.float64)
    Y = _prep(Y, np.float64)
    if Y.ndim == 1:
        Y = Y.reshape(-1, 1)
    n, p = X.shape
    r = Y.shape[1]
    w = _prep(weights, np.uint32).reshape(-1, n)
    B = w.shape[0]
    G = _empty(X, (B, p, p), np.float64)
    Bm = _empty(X, (B, p, r), np.float64)
    _check(lib().uoi_weighted_moments(_ptr(X), _ptr(Y), n, p, r, _ptr(w), B, precision, _ptr(G),
                                      _ptr(Bm), stream))
    return G, Bm


def lasso_admm_batch_noalloc(X, Y, weights, lambdas, rho=1.0, abs_tol=1e-6, rel_tol=1e-6,
                             max_iter=1000, warm_start=WARM_PATH, stream=None, out=None):
    """lasso_admm_batch without device allocation; every array must be a CUDA tensor.
    out: optional dict(beta, iters, conv) of preallocated CUDA tensors to write into
    (then this binding allocates nothing either)."""
    X = _prep(X, np.float64)
    Y = _prep(Y, np.float64)
    if Y.ndim == 1:
        Y = Y.reshape(-1, 1)
    n, p = X.shape
    r = Y.shape[1]
    lam = _prep(lambdas, np.float64)
    q = lam.shape[0]
    if weights is None:
        B, w = 1, None
    else:
        w = _prep(weights, np.uint32).reshape(-1, n)
        B = w.shape[0]
    if out is not None:
        beta, iters, conv = out["beta"], out["iters"], out["conv"]
    else:
        beta = _empty(X, (B, q, r, p), np.float64)
        iters = _empty(X, (B, q, r), np.int32)
        conv = _empty(X, (B, q, r), np.uint8)
    st = lib().lasso_admm_batch_noalloc(_ptr(X), _ptr(Y), n, p, r, _ptr(w), B, _ptr(lam), q, rho,
                                        abs_tol, rel_tol, max_iter, warm_start, _ptr(beta),
                                        _ptr(iters), _ptr(conv), stream)
    _check(st)
    return dict(beta=beta, iters=iters, conv=conv, status=st)


class WarmStartModel:
    """The learned warm-start network (device resident), see uoi_ws_* in include/uoi.h."""

    def __init__(self, seed=0, path=None):
        h = C.c_void_p()
        if path is not None:
            _check(lib().uoi_ws_load(path.encode(), C.byref(h)))
        else:
            _check(lib().uoi_ws_create(seed, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            lib().uoi_ws_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def param_count():
        return int(lib().uoi_ws_param_count())

    def get_params(self):
        out = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().uoi_ws_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().uoi_ws_set_params(self.h, a.ctypes.data))

    def forward(self, X):
        if _is_torch(X):
            import torch
            X = X.contiguous().float()
            out = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
            out = np.empty((X.shape[0], 3), dtype=np.float32)
        _check(lib().uoi_ws_forward(self.h, _ptr(X), X.shape[0], _ptr(out)))
        return out

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.empty(self.param_count(), dtype=np.float32)
        L = C.c_double()
        _check(lib().uoi_ws_loss_grad(self.h, X.ctypes.data, T.ctypes.data, X.shape[0],
                                      C.byref(L), g.ctypes.data))
        return float(L.value), g

    def train(self, X, T, epochs=10, batch=4096, lr=1e-3, seed=0):
        X = X.contiguous().float() if _is_torch(X) else np.ascontiguousarray(X, dtype=np.float32)
        T = T.contiguous().float() if _is_torch(T) else np.ascontiguousarray(T, dtype=np.float32)
        L = C.c_double()
        _check(lib().uoi_ws_train(self.h, _ptr(X), _ptr(T), X.shape[0], epochs, batch, lr, seed,
                                  C.byref(L)))
        return float(L.value)

    def save(self, path):
        _check(lib().uoi_ws_save(self.h, path.encode()))


def ws_dataset(X, Y, weights, lambdas, rho=1.0, abs_tol=1e-6, rel_tol=1e-6, max_iter=1000):
    """(features N x 8, targets N x 3) from path-warm FP64 ADMM, N = B q r p."""
    X = _prep(X, np.float64)
    Y = _prep(Y, np.float64)
    if Y.ndim == 1:
        Y = Y.reshape(-1, 1)
    n, p = X.shape
    r = Y.shape[1]
    w = _prep(weights, np.uint32).reshape(-1, n)
    B = w.shape[0]
    lam = _prep(lambdas, np.float64)
    q = lam.shape[0]
    N = B * q * r * p
    if _is_torch(X):
        import torch
        F = torch.empty((N, 8), dtype=torch.float32, device=X.device)
        T = torch.empty((N, 3), dtype=torch.float32, device=X.device)
    else:
        F = np.empty((N, 8), dtype=np.float32)
        T = np.empty((N, 3), dtype=np.float32)
    _check(lib().uoi_ws_dataset(_ptr(X), _ptr(Y), n, p, r, _ptr(w), B, _ptr(lam), q, rho, abs_tol,
                                rel_tol, max_iter, _ptr(F), _ptr(T), None))
    return F, T


def selftest_wait(limit_ns, arrive=False, stream=None):
    """Bounded mbarrier wait on the GPU (see uoi_selftest_wait); returns the
    milliseconds the wait took, raises UoiError(ERR_TIMEOUT) when it ran out."""
    ms = C.c_double(0.0)
    st = lib().uoi_selftest_wait(int(limit_ns), 1 if arrive else 0, C.byref(ms), stream)
    if st < 0:
        err = UoiError(st, last_error())
        err.waited_ms = float(ms.value)
        raise err
    return float(ms.value)


def selftest_index_check(index, extent, stream=None):
    """The device index check once (see uoi_selftest_index_check)."""
    return _check(lib().uoi_selftest_index_check(int(index), int(extent), stream))


def shutdown():
    lib().uoi_shutdown()
