"""lasso_admm_batch_noalloc: the LASSO-ADMM solver for callers that cannot allocate.

Some callers cannot let a library allocate device memory: applications that
reserve all of the device's memory at start-up for their own allocator, hosts
under a fixed device-memory quota, and latency-critical loops where an
allocation may block and a free synchronises the device.
lasso_admm_batch_noalloc works in a fixed scratch array compiled into the
library instead.

These tests call it through the C ABI, two calls in a row, for one response
(r = 1, the LASSO case) and for three, and check
  - each result against the FP64 oracle's ADMM: identical iteration counts,
    identical supports outside the 1e-6 ambiguity margin, 1e-6 relative l2 per
    column -- the bar of the other FP64 parity tests;
  - each result against the allocating entry point, lasso_admm_batch;
  - that the calls allocate nothing: the high-water mark of the device's
    default memory pool (where the library's allocations come from) and the
    device's free memory do not move, while the same measurement does see the
    allocating entry point allocate.
The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POOL_USED_HIGH = 8          # cudaMemPoolAttrUsedMemHigh


class PoolWatch:
    """High-water mark of the current device's default memory pool."""

    def __init__(self):
        native.lib()                                  # loads the CUDA runtime it links
        self.rt = C.CDLL("libcudart.so.13")
        self.pool = C.c_void_p()
        dev = torch.cuda.current_device()
        assert self.rt.cudaDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def reset(self):
        torch.cuda.synchronize()
        zero = C.c_uint64(0)                          # resets the mark to the current use
        assert self.rt.cudaMemPoolSetAttribute(self.pool, POOL_USED_HIGH, C.byref(zero)) == 0

    def high(self):
        torch.cuda.synchronize()
        v = C.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, POOL_USED_HIGH, C.byref(v)) == 0
        return int(v.value)

    def free_bytes(self):
        torch.cuda.synchronize()
        free, total = C.c_size_t(0), C.c_size_t(0)
        assert self.rt.cudaMemGetInfo(C.byref(free), C.byref(total)) == 0
        return int(free.value)


def _inputs(r=1, seed=2024):
    g = np.random.Generator(np.random.PCG64(seed))
    n, p, B, q = 200, 50, 4, 8
    X = g.standard_normal((n, p))
    Y = np.zeros((n, r))
    for e in range(r):
        beta = np.zeros(p)
        beta[g.choice(p, 10, replace=False)] = g.uniform(1, 3, 10) * g.choice([-1, 1], 10)
        Y[:, e] = X @ beta + 0.5 * g.standard_normal(n)
    w = g.integers(0, 3, size=(B, n)).astype(np.uint32)
    lmax = np.max(np.abs(X.T @ Y)) / n
    lam = lmax * np.logspace(0, -3, q)
    return X, Y, w, lam


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def _check_against_oracle(out, ref, lam, tol=1e-6):
    ob = out["beta"].cpu().numpy()
    thr = np.asarray(lam)[None, :, None, None]
    amb = (np.abs(np.abs(ref["v"]) - thr) <= tol) | ((np.abs(ref["beta"]) <= tol) & (ref["beta"] != 0))
    np.testing.assert_array_equal(out["iters"].cpu().numpy(), ref["iters"])
    assert not (((ob != 0) != (ref["beta"] != 0)) & ~amb).any()
    for idx in np.ndindex(*ob.shape[:3]):
        assert _rel(ob[idx], ref["beta"][idx]) <= tol


@pytest.mark.parametrize("r", [1, 3])
@pytest.mark.parametrize("warm", [native.WARM_PATH, native.WARM_NONE])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(warm, r):
    X, Y, w, lam = _inputs(r)
    ref = oracle.lasso_admm_batch(X, Y, w, lam, warm_start=warm)
    Xd, Yd, Wd, Ld = _dev(X), _dev(Y), _dev(w.astype(np.int32)), _dev(lam)
    alloc = native.lasso_admm_batch(Xd, Yd, Wd, Ld, warm_start=warm)
    ab = alloc["beta"].cpu().numpy()
    _check_against_oracle(alloc, ref, lam)
    for _ in range(2):
        out = native.lasso_admm_batch_noalloc(Xd, Yd, Wd, Ld, warm_start=warm)
        assert out["status"] == alloc["status"]
        _check_against_oracle(out, ref, lam)
        ob = out["beta"].cpu().numpy()
        np.testing.assert_array_equal(out["iters"].cpu().numpy(), alloc["iters"].cpu().numpy())
        assert np.array_equal(ob != 0, ab != 0)
        for idx in np.ndindex(*ab.shape[:3]):
            assert _rel(ob[idx], ab[idx]) <= 1e-6


@pytest.mark.parametrize("r", [1, 3])
def test_noalloc_allocates_nothing(r):
    X, Y, w, lam = _inputs(r, seed=77)
    Xd, Yd, Wd, Ld = _dev(X), _dev(Y), _dev(w.astype(np.int32)), _dev(lam)
    # outputs made up front, so the binding allocates nothing during the calls either
    B, q, n = w.shape[0], lam.shape[0], X.shape[0]
    outs = [dict(beta=torch.empty((B, q, r, X.shape[1]), dtype=torch.float64, device="cuda"),
                 iters=torch.empty((B, q, r), dtype=torch.int32, device="cuda"),
                 conv=torch.empty((B, q, r), dtype=torch.uint8, device="cuda")) for _ in range(2)]
    watch = PoolWatch()
    # the first call on a device does the set-up (symbol lookup, module loading)
    native.lasso_admm_batch_noalloc(Xd, Yd, Wd, Ld)
    # the measurement sees the allocating entry point allocate
    watch.reset()
    base = watch.high()
    native.lasso_admm_batch(Xd, Yd, Wd, Ld)
    assert watch.high() > base
    # ... and sees nothing from two calls in a row of the allocation-free one
    watch.reset()
    base, free0 = watch.high(), watch.free_bytes()
    for o in outs:
        st = native.lasso_admm_batch_noalloc(Xd, Yd, Wd, Ld, out=o)["status"]
        assert st in (native.OK, native.OK_WITH_WARNINGS)
    assert watch.high() == base
    assert watch.free_bytes() == free0
    np.testing.assert_array_equal(outs[0]["beta"].cpu().numpy(), outs[1]["beta"].cpu().numpy())


def test_noalloc_rejects_host_memory_and_oversize():
    X, Y, w, lam = _inputs()
    with pytest.raises(native.UoiError) as ei:
        native.lasso_admm_batch_noalloc(X, Y, w, lam)
    assert ei.value.status == native.ERR_INVALID_ARG
    big = torch.zeros((300, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(native.UoiError) as ei:
        native.lasso_admm_batch_noalloc(big, torch.zeros((300, 1), dtype=torch.float64, device="cuda"),
                                        None, _dev(lam))
    assert ei.value.status == native.ERR_INVALID_ARG
    assert "UOI_NOALLOC_MAX_P" in native.last_error()
    # within the p limit but beyond the 16 MiB array: B = 64 weight vectors at p = 128
    n, p, B = 256, 128, 64
    Xb = torch.zeros((n, p), dtype=torch.float64, device="cuda")
    Wb = torch.ones((B, n), dtype=torch.int32, device="cuda")
    with pytest.raises(native.UoiError) as ei:
        native.lasso_admm_batch_noalloc(Xb, torch.zeros((n, 1), dtype=torch.float64, device="cuda"),
                                        Wb, _dev(lam))
    assert ei.value.status == native.ERR_INVALID_ARG
    assert "16 MiB" in native.last_error()
