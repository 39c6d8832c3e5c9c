"""lasso_admm_batch_noalloc: the solver variant for callers that cannot allocate.

Some callers must not let a library allocate device memory (allocation-free
stream captures, applications that own all device memory, latency-critical
loops).  lasso_admm_batch_noalloc works in a fixed scratch array compiled into
the library instead.  This test calls it through the C ABI twice in a row and
checks each result against the allocating entry point, lasso_admm_batch, with
the tolerance of the other parity tests (1e-6 relative l2 per column,
identical supports and iteration counts).  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

from paper_1808_06992_gb300 import native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs():
    g = np.random.Generator(np.random.PCG64(2024))
    n, p, B, q = 200, 50, 4, 8
    X = g.standard_normal((n, p))
    beta = np.zeros(p)
    beta[g.choice(p, 10, replace=False)] = g.uniform(1, 3, 10) * g.choice([-1, 1], 10)
    y = X @ beta + 0.5 * g.standard_normal(n)
    w = g.integers(0, 3, size=(B, n)).astype(np.uint32)
    lmax = np.max(np.abs(X.T @ y)) / n
    lam = lmax * np.logspace(0, -3, q)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(X), dev(y.reshape(-1, 1)), dev(w.astype(np.int32)), dev(lam)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


@pytest.mark.parametrize("warm", [native.WARM_PATH, native.WARM_NONE])
def test_noalloc_matches_allocating_entry_point_twice(warm):
    X, Y, W, lam = _inputs()
    ref = native.lasso_admm_batch(X, Y, W, lam, warm_start=warm)
    rb = ref["beta"].cpu().numpy()
    for _ in range(2):
        out = native.lasso_admm_batch_noalloc(X, Y, W, lam, warm_start=warm)
        ob = out["beta"].cpu().numpy()
        assert out["status"] == ref["status"]
        np.testing.assert_array_equal(out["iters"].cpu().numpy(), ref["iters"].cpu().numpy())
        assert np.array_equal(ob != 0, rb != 0)
        for idx in np.ndindex(*rb.shape[:3]):
            assert _rel(ob[idx], rb[idx]) <= 1e-6


def test_noalloc_rejects_host_memory_and_oversize():
    X, Y, W, lam = _inputs()
    with pytest.raises(native.UoiError) as ei:
        native.lasso_admm_batch_noalloc(X.cpu().numpy(), Y.cpu().numpy(), W.cpu().numpy(),
                                        lam.cpu().numpy())
    assert ei.value.status == native.ERR_INVALID_ARG
    big = torch.zeros((300, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(native.UoiError) as ei:
        native.lasso_admm_batch_noalloc(big, Y[:300] if Y.shape[0] >= 300 else
                                        torch.zeros((300, 1), dtype=torch.float64, device="cuda"),
                                        None, lam)
    assert ei.value.status == native.ERR_INVALID_ARG
    assert "UOI_NOALLOC_MAX_P" in native.last_error()
