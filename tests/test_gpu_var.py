"""VAR(d) lagged design and the unpenalised intercept: CUDA path vs the FP64
oracle through the C ABI (GPU).  Same bars as the other parity tests: bit-exact
indices and supports (ambiguous features excluded), 1e-6 relative l2 on the
coefficients in the plain FP64 form, 1e-5 in the mixed form (Alg. 2, Eq. 6-9)."""
import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import native, synth

from test_gpu_parity import bits_to_bool, compare_fit, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def lagged(S, d):
    """Eq. 7-8 by slicing: Y = rows d.., X = (rows d-1.., ..., rows 0..)."""
    N = S.shape[0]
    X = np.concatenate([S[d - j:N - j] for j in range(1, d + 1)], axis=1)
    return np.ascontiguousarray(X), np.ascontiguousarray(S[d:])


@pytest.mark.parametrize("order", [1, 2, 3])
def test_lagged_intercept_full_trace_fp64(order):
    v = synth.var_d_problem(10, 300, order, 0.15, 0.85, seed=50 + order, mu_scale=2.0, burn_in=100)
    X, Y = lagged(v.series, order)
    kw = dict(B1=5, B2=4, q=8, block_len=20, intercept=1)
    ref = oracle.uoi_fit(X, Y, **kw)
    gpu = native.uoi_fit_traced(X, Y, precision=native.PREC_FP64, **kw)
    assert gpu["beta"].shape == (10, 10 * order + 1)
    rep = compare_fit(ref, gpu, X, Y, **kw)
    assert rep["family_clean"]


@pytest.mark.parametrize("order,icpt", [(2, 1), (3, 0), (1, 1)])
def test_var_fit_order_and_intercept_fp64(order, icpt):
    v = synth.var_d_problem(12, 400, order, 0.1, 0.8, seed=60 + order, mu_scale=1.5, burn_in=100)
    kw = dict(B1=5, B2=4, q=8, block_len=25, intercept=icpt)
    ref = oracle.uoi_var_fit(v.series, order=order, **kw)
    out = native.uoi_var_fit(v.series, order=order, **kw)
    assert out["A"].shape == (order, 12, 12)
    assert rel_l2(out["A"], ref["A"]) <= 1e-6
    if icpt:
        assert rel_l2(out["mu"], ref["mu"]) <= 1e-6
    else:
        assert np.all(out["mu"] == 0)
    # the entry point's own design equals the traced fit on the sliced design
    X, Y = lagged(v.series, order)
    tr = native.uoi_fit_traced(X, Y, **kw)
    np.testing.assert_array_equal(out["A"], tr["beta"][:, :order * 12].reshape(12, order, 12).transpose(1, 0, 2))
    if icpt:
        np.testing.assert_array_equal(out["mu"], tr["beta"][:, -1])


def test_var_fit_device_pointers():
    v = synth.var_d_problem(8, 200, 2, 0.2, 0.8, seed=70, mu_scale=1.0, burn_in=50)
    kw = dict(B1=3, B2=3, q=5, block_len=10, intercept=1)
    host = native.uoi_var_fit(v.series, order=2, **kw)
    dev = native.uoi_var_fit(torch.from_numpy(v.series).cuda(), order=2, **kw)
    assert dev["A"].is_cuda and dev["mu"].is_cuda
    np.testing.assert_array_equal(dev["A"].cpu().numpy(), host["A"])
    np.testing.assert_array_equal(dev["mu"].cpu().numpy(), host["mu"])


def test_intercept_large_column_means_fp64():
    # columns far from zero mean: centring before the Gram keeps the elimination exact
    d = synth.lasso_problem(400, 40, 6, seed=71, sigma=0.5)
    X = d.X + np.linspace(-50, 80, 40)
    y = d.y + 25.0
    kw = dict(B1=5, B2=4, q=8, intercept=1)
    ref = oracle.uoi_fit(X, y[:, None], **kw)
    gpu = native.uoi_fit_traced(X, y, **kw)
    compare_fit(ref, gpu, X, y[:, None], **kw)


@pytest.mark.parametrize("order", [1, 2])
def test_var_intercept_mixed_within_1e5(order):
    # mixed form: tensor-core Gram of [X~ 1], FP32 ADMM, refined OLS
    v = synth.var_d_problem(48, 2000, order, 0.05, 0.85, seed=80 + order, mu_scale=2.0, burn_in=200)
    kw = dict(B1=6, B2=5, q=10, block_len=50, intercept=1)
    ref = oracle.uoi_var_fit(v.series, order=order, n_threads=6, **kw)
    out = native.uoi_var_fit(v.series, order=order, precision=native.PREC_MIXED, **kw)
    X, Y = lagged(v.series, order)
    tr = native.uoi_fit_traced(X, Y, precision=native.PREC_MIXED, **kw)
    P = 48 * order
    fam_g = bits_to_bool(tr["family"], P)
    fam_r = bits_to_bool(ref["family"], P)
    assert (fam_g != fam_r).sum() == 0
    np.testing.assert_array_equal(tr["est_jstar"], ref["est_jstar"])
    assert rel_l2(out["A"], ref["A"]) <= 1e-5
    assert rel_l2(out["mu"], ref["mu"]) <= 1e-5


def test_var_intercept_tensor_core_xupdate_mixed():
    # P = 2 p = 200 > 192: the tensor-core x-update runs on the eliminated moments;
    # checked on what is unique: bagged A and mu against the oracle
    v = synth.var_d_problem(100, 1500, 2, 0.02, 0.8, seed=90, mu_scale=1.0, burn_in=200)
    kw = dict(B1=2, B2=2, q=4, block_len=100, intercept=1)
    ref = oracle.uoi_var_fit(v.series, order=2, n_threads=2, **kw)
    out = native.uoi_var_fit(v.series, order=2, precision=native.PREC_MIXED, **kw)
    assert rel_l2(out["A"], ref["A"]) <= 1e-5
    assert rel_l2(out["mu"], ref["mu"]) <= 1e-5


@pytest.mark.parametrize("p,order,N", [(1, 2, 40), (5, 3, 15)])
def test_var_small_and_short_series_fp64(p, order, N):
    # one channel, and a series only a few rows longer than the order
    v = synth.var_d_problem(p, N, order, 0.5, 0.7, seed=100 + p, mu_scale=1.0, burn_in=30)
    kw = dict(B1=4, B2=3, q=6, intercept=1)
    ref = oracle.uoi_var_fit(v.series, order=order, **kw)
    out = native.uoi_var_fit(v.series, order=order, **kw)
    assert ref["status"] >= 0
    assert rel_l2(out["A"], ref["A"]) <= 1e-6
    assert rel_l2(out["mu"], ref["mu"]) <= 1e-6


@pytest.mark.parametrize("order,icpt", [(1, 0), (2, 1)])
def test_moving_block_bootstrap_full_trace_fp64(order, icpt):
    # moving (overlapping) selection blocks: weights bit-exact, then the whole trace
    v = synth.var_d_problem(10, 300, order, 0.15, 0.85, seed=110 + order, mu_scale=1.0, burn_in=100)
    X, Y = lagged(v.series, order)
    kw = dict(B1=5, B2=4, q=8, block_len=23, intercept=icpt, block_mode=1)
    ref = oracle.uoi_fit(X, Y, **kw)
    gpu = native.uoi_fit_traced(X, Y, precision=native.PREC_FP64, **kw)
    rep = compare_fit(ref, gpu, X, Y, **kw)
    assert rep["family_clean"]
    fixed = native.uoi_fit_traced(X, Y, precision=native.PREC_FP64, **dict(kw, block_mode=0))
    assert not np.array_equal(fixed["sel_weights"], gpu["sel_weights"])
