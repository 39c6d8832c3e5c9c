"""FP64 CPU oracle for the UoI_LASSO / UoI_VAR(d) hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The CUDA library
never imports, links or runs it, and the two share no code: the oracle is
plain C (``uoi_oracle.c``) written from the paper (arXiv 1808.06992, Alg. 1-2,
Eq. 1-9) plus Philox4x64-10 (Salmon et al., SC'11), loaded here with ctypes.

Parity status: every stage function is pinned by ``tests/test_oracle_pins.py``
(``kkt_polish``, ``kkt_residual`` and the bounds by ``tests/test_oracle_kkt.py``)
(numpy Philox, closed forms, KKT, lambda_max, brute force over supports,
sklearn, lstsq, brute-force set logic).  ``uoi_fit`` as a whole is pinned
through those parts, the noiseless recovery special case, the cases whose
selection is decided in advance, and the general case on LASSO (with and
without an intercept) and VAR(1) fixtures with varying supports (``tests/test_oracle_whole_fit.py``: selection by
scikit-learn's LASSO on the bootstrap rows repeated by multiplicity, then
intersection, least squares on the training draws, held-out losses, argmin and
median by numpy, with the fixtures' KKT margins asserted).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, OK_WITH_WARNINGS = 0, 1
ERR_INVALID_ARG, ERR_NONFINITE, ERR_NOT_PD, ERR_UNSUPPORTED = -1, -2, -3, -8
TAG_SELECTION, TAG_SPLIT, TAG_RESAMPLE = 1, 2, 3


def build_oracle(force: bool = False) -> str:
    """Compile uoi_oracle.c into oracle/_build/liboracle.so with gcc (-fopenmp)."""
    src = os.path.join(_HERE, "uoi_oracle.c")
    hdr = os.path.join(_HERE, "uoi_oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class RefParams(C.Structure):
    _fields_ = [
        ("B1", C.c_int32), ("B2", C.c_int32), ("q", C.c_int32),
        ("lambdas", C.POINTER(C.c_double)),
        ("lambda_min_ratio", C.c_double),
        ("rho", C.c_double), ("abs_tol", C.c_double), ("rel_tol", C.c_double),
        ("max_iter", C.c_int32),
        ("train_frac", C.c_double),
        ("seed", C.c_uint64), ("problem_id", C.c_uint64),
        ("block_len", C.c_int64),
        ("bagging", C.c_int32), ("split_fixed", C.c_int32), ("warm_start", C.c_int32),
        ("n_threads", C.c_int32),
        ("intercept", C.c_int32), ("block_mode", C.c_int32),
    ]


class RefTrace(C.Structure):
    _fields_ = [
        ("lambdas", C.POINTER(C.c_double)),
        ("sel_beta", C.POINTER(C.c_double)),
        ("sel_v", C.POINTER(C.c_double)),
        ("sel_iters", C.POINTER(C.c_int32)),
        ("sel_conv", C.POINTER(C.c_uint8)),
        ("family", C.POINTER(C.c_uint64)),
        ("est_beta", C.POINTER(C.c_double)),
        ("est_loss", C.POINTER(C.c_double)),
        ("est_jstar", C.POINTER(C.c_int32)),
        ("est_fallback", C.POINTER(C.c_int32)),
        ("eval_count", C.POINTER(C.c_int32)),
    ]


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build_oracle())
            d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int32, C.c_uint64
            P = C.POINTER
            L.ref_philox4x64_10.argtypes = [P(u64), P(u64), P(u64)]
            L.ref_draw.argtypes = [u64, u64, u64, u64, u64]
            L.ref_draw.restype = u64
            L.ref_range_map.argtypes = [u64, u64]
            L.ref_range_map.restype = u64
            L.ref_selection_weights.argtypes = [i64, i64, u64, u64, i64, P(C.c_uint32)]
            L.ref_selection_weights_moving.argtypes = [i64, i64, u64, u64, i64, P(C.c_uint32)]
            L.ref_estimation_weights.argtypes = [i64, i64, d, C.c_int, u64, u64, i64,
                                                 P(C.c_uint32), P(C.c_uint8), P(i64)]
            L.ref_weighted_moments.argtypes = [P(d), i64, P(d), i64, i64, i64, i64,
                                               P(C.c_uint32), P(d), P(d), P(d)]
            L.ref_cholesky.argtypes = [P(d), i64, P(d)]
            L.ref_cholesky_solve.argtypes = [P(d), i64, P(d), P(d)]
            L.ref_lambda_max.argtypes = [P(d), i64, P(d), i64, i64, i64, i64]
            L.ref_lambda_max.restype = d
            L.ref_lambda_grid.argtypes = [d, i32, d, P(d)]
            L.ref_admm_column.argtypes = [P(d), P(d), i64, d, d, d, d, i32,
                                          P(d), P(d), P(d), P(d), P(i32)]
            L.ref_lasso_admm_batch.argtypes = [P(d), i64, P(d), i64, i64, i64, i64,
                                               P(C.c_uint32), i32, P(d), i32, d, d, d, i32, i32,
                                               P(i64), i64, P(d), P(i32), P(C.c_uint8), P(d)]
            L.ref_ols_support.argtypes = [P(d), P(d), i64, i64, P(u64), P(d)]
            L.ref_kkt_polish.argtypes = [P(d), P(d), i64, i64, d, d, P(d), i32, P(d), P(d), P(i32)]
            L.ref_lasso_admm_intercept.argtypes = [P(d), i64, P(d), i64, i64, i64, i64,
                                                   P(C.c_uint32), P(d), i32, d, d, d, i32, i32,
                                                   P(d), P(d), P(i32), P(C.c_uint8), P(d)]
            L.ref_lagged_design.argtypes = [P(d), i64, i64, i32, P(d), P(d)]
            L.ref_uoi_var_fit.argtypes = [P(d), i64, i64, i32, P(RefParams), P(d), P(d),
                                          P(RefTrace)]
            L.ref_uoi_fit.argtypes = [P(d), i64, P(d), i64, i64, i64, i64,
                                      P(RefParams), P(d), P(RefTrace)]
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# numpy-facing wrappers
# ----------------------------------------------------------------------------
def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().ref_philox4x64_10(_p(c, C.c_uint64), _p(k, C.c_uint64), _p(out, C.c_uint64))
    return out


def draw(seed, problem, k, tag, i):
    return int(lib().ref_draw(seed, problem, k, tag, i))


def range_map(r, n):
    return int(lib().ref_range_map(r, n))


def selection_weights(m, block_len, seed, problem, k):
    w = np.zeros(m, dtype=np.uint32)
    lib().ref_selection_weights(m, block_len, seed, problem, k, _p(w, C.c_uint32))
    return w


def selection_weights_moving(m, block_len, seed, problem, k):
    w = np.zeros(m, dtype=np.uint32)
    lib().ref_selection_weights_moving(m, block_len, seed, problem, k, _p(w, C.c_uint32))
    return w


def estimation_weights(m, block_len, train_frac, split_fixed, seed, problem, k):
    L = max(int(block_len), 1)
    units = (m + L - 1) // L
    w = np.zeros(m, dtype=np.uint32)
    ev = np.zeros(m, dtype=np.uint8)
    perm = np.zeros(units, dtype=np.int64)
    st = lib().ref_estimation_weights(m, block_len, train_frac, int(split_fixed), seed, problem,
                                      k, _p(w, C.c_uint32), _p(ev, C.c_uint8),
                                      _p(perm, C.c_int64))
    if st != 0:
        raise ValueError(f"estimation split failed: {st}")
    return w, ev, perm


def weighted_moments(X, Y, w=None, want_yy=False):
    X = _f64(X)
    Y = _f64(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    m, p = X.shape
    r = Y.shape[1]
    G = np.zeros((p, p))
    B = np.zeros((p, r))
    yy = np.zeros(r) if want_yy else None
    wa = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
    lib().ref_weighted_moments(_p(X, C.c_double), p, _p(Y, C.c_double), r, m, p, r,
                               _p(wa, C.c_uint32), _p(G, C.c_double), _p(B, C.c_double),
                               _p(yy, C.c_double))
    return (G, B, yy) if want_yy else (G, B)


def cholesky(A):
    A = _f64(A)
    p = A.shape[0]
    L = np.zeros((p, p))
    st = lib().ref_cholesky(_p(A, C.c_double), p, _p(L, C.c_double))
    return L, int(st)


def cholesky_solve(L, b):
    L = _f64(L)
    b = _f64(b)
    x = np.zeros_like(b)
    lib().ref_cholesky_solve(_p(L, C.c_double), L.shape[0], _p(b, C.c_double), _p(x, C.c_double))
    return x


def lambda_max(X, Y):
    X = _f64(X)
    Y = _f64(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    m, p = X.shape
    return float(lib().ref_lambda_max(_p(X, C.c_double), p, _p(Y, C.c_double), Y.shape[1],
                                      m, p, Y.shape[1]))


def lambda_grid(lmax, q, ratio=1e-3):
    out = np.zeros(q)
    lib().ref_lambda_grid(lmax, q, ratio, _p(out, C.c_double))
    return out


def admm_column(L, bn, lam, rho=1.0, abs_tol=1e-6, rel_tol=1e-6, max_iter=1000, z0=None, u0=None):
    L = _f64(L)
    bn = _f64(bn)
    p = bn.shape[0]
    z = np.zeros(p) if z0 is None else _f64(z0).copy()
    u = np.zeros(p) if u0 is None else _f64(u0).copy()
    x = np.zeros(p)
    v = np.zeros(p)
    it = C.c_int32(0)
    conv = lib().ref_admm_column(_p(L, C.c_double), _p(bn, C.c_double), p, lam, rho, abs_tol,
                                 rel_tol, max_iter, _p(z, C.c_double), _p(u, C.c_double),
                                 _p(x, C.c_double), _p(v, C.c_double), C.byref(it))
    return dict(z=z, u=u, x=x, v=v, iters=int(it.value), converged=bool(conv))


def lasso_admm_batch(X, Y, weights, lambdas, rho=1.0, abs_tol=1e-6, rel_tol=1e-6, max_iter=1000,
                     warm_start=1, eq_list=None):
    """Returns dict(beta (B,q,r,p), iters, conv, v, status)."""
    X = _f64(X)
    Y = _f64(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    m, p = X.shape
    r = Y.shape[1]
    lam = _f64(lambdas)
    q = lam.shape[0]
    if weights is None:
        B = 1
        wa = None
    else:
        wa = np.ascontiguousarray(weights, dtype=np.uint32).reshape(-1, m)
        B = wa.shape[0]
    eq = None if eq_list is None else np.ascontiguousarray(eq_list, dtype=np.int64)
    re = r if eq is None else eq.shape[0]
    beta = np.zeros((B, q, re, p))
    v = np.zeros((B, q, re, p))
    iters = np.zeros((B, q, re), dtype=np.int32)
    conv = np.zeros((B, q, re), dtype=np.uint8)
    st = lib().ref_lasso_admm_batch(_p(X, C.c_double), p, _p(Y, C.c_double), r, m, p, r,
                                    _p(wa, C.c_uint32), B, _p(lam, C.c_double), q, rho, abs_tol,
                                    rel_tol, max_iter, warm_start, _p(eq, C.c_int64),
                                    0 if eq is None else re, _p(beta, C.c_double),
                                    _p(iters, C.c_int32), _p(conv, C.c_uint8), _p(v, C.c_double))
    return dict(beta=beta, iters=iters, conv=conv.astype(bool), v=v, status=int(st))


def lasso_admm_intercept(X, Y, weights, lambdas, rho=1.0, abs_tol=1e-6, rel_tol=1e-6,
                         max_iter=1000, warm_start=1):
    """LASSO with an unpenalised intercept for one weight vector (or None).
    Returns dict(beta (q,r,p), mu (q,r), iters, conv, v, status)."""
    X = _f64(X)
    Y = _f64(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    m, p = X.shape
    r = Y.shape[1]
    lam = _f64(lambdas)
    q = lam.shape[0]
    wa = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32).reshape(m)
    beta = np.zeros((q, r, p))
    mu = np.zeros((q, r))
    v = np.zeros((q, r, p))
    iters = np.zeros((q, r), dtype=np.int32)
    conv = np.zeros((q, r), dtype=np.uint8)
    st = lib().ref_lasso_admm_intercept(_p(X, C.c_double), p, _p(Y, C.c_double), r, m, p, r,
                                        _p(wa, C.c_uint32), _p(lam, C.c_double), q, rho, abs_tol,
                                        rel_tol, max_iter, warm_start, _p(beta, C.c_double),
                                        _p(mu, C.c_double), _p(iters, C.c_int32),
                                        _p(conv, C.c_uint8), _p(v, C.c_double))
    return dict(beta=beta, mu=mu, iters=iters, conv=conv.astype(bool), v=v, status=int(st))


def lagged_design(series, order):
    """(X, Y) of Eq. 7-8 for a VAR(order), rows in ascending time."""
    S = _f64(series)
    N, p = S.shape
    X = np.zeros((N - order, order * p))
    Y = np.zeros((N - order, p))
    lib().ref_lagged_design(_p(S, C.c_double), N, p, order, _p(X, C.c_double), _p(Y, C.c_double))
    return X, Y


def ols_support(G, b, support_bits):
    G = _f64(G)
    b = _f64(b).reshape(-1)
    p = G.shape[0]
    S = np.ascontiguousarray(support_bits, dtype=np.uint64)
    beta = np.zeros(p)
    fb = lib().ref_ols_support(_p(G, C.c_double), _p(b, C.c_double), 1, p, _p(S, C.c_uint64),
                               _p(beta, C.c_double))
    return beta, bool(fb)


def kkt_polish(G, b, nk, lam, z_start, max_moves=None):
    """Exact minimiser of (1/2nk)||y - X beta||_W^2 + lam ||beta||_1 from the support
    and signs of z_start (ref_kkt_polish).  G = X^T W X, b = X^T W y.
    Returns dict(beta, grad (= (b - G beta)/nk), certified, moves, status)."""
    G = _f64(G)
    b = _f64(b).reshape(-1)
    z = _f64(z_start).reshape(-1)
    p = G.shape[0]
    beta = np.zeros(p)
    grad = np.zeros(p)
    mv = C.c_int32(0)
    st = lib().ref_kkt_polish(_p(G, C.c_double), _p(b, C.c_double), 1, p, float(nk), float(lam),
                              _p(z, C.c_double), int(4 * p if max_moves is None else max_moves),
                              _p(beta, C.c_double), _p(grad, C.c_double), C.byref(mv))
    return dict(beta=beta, grad=grad, certified=st == 0, moves=int(mv.value), status=int(st))


def kkt_residual(G, b, nk, lam, z):
    """dist(0, dF(z)) for F(beta) = (1/2) beta^T H beta - c^T beta + lam ||beta||_1,
    H = G/nk, c = b/nk: the smallest ||c - H z - s|| over s in lam d||z||_1
    (s_i = lam sign z_i where z_i != 0, s_i = clip(g_i, -lam, lam) elsewhere).
    Any z is the exact minimiser of F - xi^T beta for some xi of this norm."""
    H = _f64(G) / nk
    g = _f64(b).reshape(-1) / nk - H @ _f64(z)
    on = z != 0
    xi = np.where(on, g - lam * np.sign(z), g - np.clip(g, -lam, lam))
    return float(np.linalg.norm(xi))


def admm_stop_bound(H_norm, p, z, lam, rho=1.0, abs_tol=1e-6, rel_tol=1e-6, eta=0.0, c_norm=0.0):
    """Bound on kkt_residual of an ADMM iterate z that met the stopping rule of Eq. 5
    (primal ||x - z|| <= eps_pri, dual rho ||z - z_prev|| <= eps_dual).  At the stop
    c - H z - rho u = H (x - z) + rho (z - z_prev) with rho u in lam d||z||_1, so the
    residual is at most ||H|| eps_pri + eps_dual; eps_pri uses ||x|| <= ||z|| + eps_pri
    and eps_dual uses rho ||u|| <= lam sqrt(p) (|rho u_i| <= lam).  eta > 0 adds
    arithmetic that is accurate to eta relative (x-update, moments):
    eta ((||H|| + rho) (||z|| + eps_pri) + ||c||)."""
    zn = float(np.linalg.norm(z))
    sp = np.sqrt(p)
    eps_pri = (sp * abs_tol + rel_tol * zn) / (1.0 - rel_tol)
    eps_dual = sp * abs_tol + rel_tol * lam * sp
    return H_norm * eps_pri + eps_dual + eta * ((H_norm + rho) * (zn + eps_pri) + c_norm)


def support_band(beta_hat, grad_hat, lam, kappa, mu, H_norm):
    """Features whose membership in the support of a point with kkt_residual <= kappa
    is not decided by the exact minimiser beta_hat (gradient grad_hat): such a point z
    satisfies ||z - beta_hat|| <= kappa / mu (mu = smallest eigenvalue of H), so
    |beta_hat_i| > kappa / mu forces z_i != 0 with the same sign, and
    |grad_hat_i| < lam - kappa (1 + ||H|| / mu) forces z_i = 0."""
    delta = kappa / mu
    on = beta_hat != 0
    return (on & (np.abs(beta_hat) <= delta)) | (~on & (lam - np.abs(grad_hat) <= kappa + H_norm * delta))


def make_params(B1, B2, q, lambdas=None, lambda_min_ratio=1e-3, rho=1.0, abs_tol=1e-6,
                rel_tol=1e-6, max_iter=1000, train_frac=0.8, seed=0, problem_id=0, block_len=0,
                bagging=0, split_fixed=0, warm_start=1, n_threads=1, intercept=0, block_mode=0):
    keep = None
    prm = RefParams()
    prm.B1, prm.B2, prm.q = B1, B2, q
    if lambdas is not None:
        keep = _f64(lambdas)
        prm.lambdas = _p(keep, C.c_double)
    prm.lambda_min_ratio = lambda_min_ratio
    prm.rho, prm.abs_tol, prm.rel_tol = rho, abs_tol, rel_tol
    prm.max_iter = max_iter
    prm.train_frac = train_frac
    prm.seed, prm.problem_id = seed, problem_id
    prm.block_len = block_len
    prm.bagging, prm.split_fixed, prm.warm_start = bagging, split_fixed, warm_start
    prm.n_threads = n_threads
    prm.intercept = int(bool(intercept))
    prm.block_mode = int(block_mode)
    return prm, keep


def uoi_fit(X, Y, B1, B2, q, trace=True, **kw):
    """Full UoI fit of the responses Y (m x r) on X (m x p).

    Returns dict(beta (r, pa), status, and the trace arrays when trace=True);
    pa = p + 1 with an intercept (the last column is mu), else p."""
    X = _f64(X)
    Y = _f64(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    m, p = X.shape
    r = Y.shape[1]
    W = (p + 63) // 64
    prm, keep = make_params(B1, B2, q, **kw)
    pa = p + prm.intercept
    beta = np.zeros((r, pa))
    out = dict()
    tr = None
    if trace:
        out = dict(
            lambdas=np.zeros(q), sel_beta=np.zeros((B1, q, r, p)), sel_v=np.zeros((B1, q, r, p)),
            sel_iters=np.zeros((B1, q, r), dtype=np.int32),
            sel_conv=np.zeros((B1, q, r), dtype=np.uint8),
            family=np.zeros((q, r, W), dtype=np.uint64), est_beta=np.zeros((B2, q, r, pa)),
            est_loss=np.zeros((B2, q, r)), est_jstar=np.zeros(B2, dtype=np.int32),
            est_fallback=np.zeros((B2, q, r), dtype=np.int32),
            eval_count=np.zeros(B2, dtype=np.int32))
        tr = RefTrace()
        for name, ct in RefTrace._fields_:
            setattr(tr, name, _p(out[name], ct._type_))
    st = lib().ref_uoi_fit(_p(X, C.c_double), p, _p(Y, C.c_double), r, m, p, r, C.byref(prm),
                           _p(beta, C.c_double), C.byref(tr) if tr is not None else None)
    del keep
    out["beta"] = beta
    out["status"] = int(st)
    return out


def uoi_lasso_fit(X, y, B1, B2, q, **kw):
    return uoi_fit(X, np.asarray(y).reshape(-1, 1), B1, B2, q, **kw)


def uoi_var_fit(series, B1, B2, q, order=1, **kw):
    """VAR(order) (Alg. 2, Eq. 6-9): the lagged design of ``lagged_design``
    fitted as p LASSOs sharing it, then beta* partitioned into A (order, p, p),
    A[j-1][e, i] = coefficient of X_{t-j,i} in equation e, and mu (p)."""
    X, Y = lagged_design(series, order)
    out = uoi_fit(X, Y, B1, B2, q, **kw)
    p = Y.shape[1]
    b = out["beta"]
    out["A"] = b[:, :order * p].reshape(p, order, p).transpose(1, 0, 2).copy()
    out["mu"] = b[:, order * p].copy() if b.shape[1] > order * p else np.zeros(p)
    return out


def uoi_var_fit_c(series, B1, B2, q, order=1, **kw):
    """The same fit through the C entry point, which builds the design and
    partitions beta* itself.  Returns (A, mu, status)."""
    S = _f64(series)
    N, p = S.shape
    prm, keep = make_params(B1, B2, q, **kw)
    A = np.zeros((max(order, 1), p, p))
    mu = np.zeros(p)
    st = lib().ref_uoi_var_fit(_p(S, C.c_double), N, p, order, C.byref(prm), _p(A, C.c_double),
                               _p(mu, C.c_double), None)
    del keep
    return A, mu, int(st)
