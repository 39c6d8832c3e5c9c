"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU).

Tolerances (plain FP64 form): bootstrap indices, supports, family and j* are
bit-exact (features within 1e-6 of the soft-threshold are excluded and
counted); coefficients agree within 1e-6 relative l2 per column.  The mixed
form (FP32 ADMM) is held to 1e-5 relative l2 on the bagged estimate.
"""
import numpy as np
import pytest

import mixed_check
import oracle
from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def ambiguous(ref, lam, rho=1.0, tol=1e-6):
    """Features within tol of the zero threshold in the oracle's final iterate."""
    thr = np.asarray(lam)[None, :, None, None] / rho
    v, z = ref["sel_v"], ref["sel_beta"]
    return (np.abs(np.abs(v) - thr) <= tol) | ((np.abs(z) <= tol) & (z != 0))


def bits_to_bool(words, p):
    w = np.asarray(words).astype(np.uint64)
    out = np.zeros(w.shape[:-1] + (p,), dtype=bool)
    for i in range(p):
        out[..., i] = (w[..., i // 64] >> np.uint64(i % 64)) & np.uint64(1)
    return out


def compare_fit(ref, gpu, X, Y, lam_tol=1e-13, coef_tol=1e-6, check_weights=True, **kw):
    """Full-trace comparison of an oracle fit and a GPU fit on the same inputs."""
    B1, q, r, p = ref["sel_beta"].shape
    m = X.shape[0]
    report = {}
    # lambda grid
    assert rel_l2(gpu["lambdas"], ref["lambdas"]) <= lam_tol
    # bootstrap indices: bit-exact
    if check_weights:
        blk = kw.get("block_len", 0)
        sel = oracle.selection_weights_moving if kw.get("block_mode", 0) == 1 else oracle.selection_weights
        for k in range(B1):
            want = sel(m, blk, kw.get("seed", 0), kw.get("problem_id", 0), k)
            np.testing.assert_array_equal(gpu["sel_weights"][k], want)
        B2 = ref["est_loss"].shape[0]
        for k in range(B2):
            w, ev, _ = oracle.estimation_weights(m, blk, kw.get("train_frac", 0.8),
                                                 kw.get("split_mode", 0), kw.get("seed", 0),
                                                 kw.get("problem_id", 0), k)
            np.testing.assert_array_equal(gpu["est_weights"][k], w)
            np.testing.assert_array_equal(gpu["est_eval"][k], ev)
    # selection estimates and supports
    amb = ambiguous(ref, ref["lambdas"])
    report["ambiguous"] = int(amb.sum())
    gs = gpu["sel_beta"] != 0
    rs = ref["sel_beta"] != 0
    mism = (gs != rs) & ~amb
    assert mism.sum() == 0, f"{int(mism.sum())} support bits differ"
    np.testing.assert_array_equal(gpu["sel_iters"], ref["sel_iters"])
    errs = [rel_l2(gpu["sel_beta"][k, j, e], ref["sel_beta"][k, j, e])
            for k in range(B1) for j in range(q) for e in range(r)]
    report["sel_max_rel"] = float(np.max(errs))
    assert report["sel_max_rel"] <= coef_tol
    # family (Eq. 3)
    fam_g = bits_to_bool(gpu["family"], p)
    fam_r = bits_to_bool(ref["family"], p)
    touched = amb.any(axis=0)
    assert np.array_equal(fam_g | touched, fam_r | touched)
    clean = not (fam_g != fam_r).any()
    if clean:
        np.testing.assert_allclose(gpu["est_loss"], ref["est_loss"], rtol=1e-9, atol=1e-12)
        np.testing.assert_array_equal(gpu["est_jstar"], ref["est_jstar"])
        B2 = ref["est_loss"].shape[0]
        for k in range(B2):
            j = ref["est_jstar"][k]
            for e in range(r):
                assert rel_l2(gpu["est_beta"][k, e], ref["est_beta"][k, j, e]) <= coef_tol
        report["beta_rel"] = rel_l2(gpu["beta"], ref["beta"])
        assert report["beta_rel"] <= coef_tol
    report["family_clean"] = clean
    return report


def iteration_histogram(iters, conv):
    """uoi_diag.admm_iter_hist from per-column iteration counts and flags."""
    it = np.asarray(iters).ravel()
    cv = np.asarray(conv).ravel().astype(bool)
    edges = [16, 32, 64, 128, 256, 512]
    h = [int(np.sum(cv & (it <= edges[0])))]
    h += [int(np.sum(cv & (it > lo) & (it <= hi))) for lo, hi in zip(edges[:-1], edges[1:])]
    h += [int(np.sum(cv & (it > edges[-1]))), int(np.sum(~cv))]
    return h


def test_c1_fp64_parity_full_trace():
    d = synth.workload_data(1)
    kw = dict(B1=20, B2=10, q=16)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, precision=native.PREC_FP64, **kw)
    rep = compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), **kw)
    assert rep["family_clean"]
    assert gpu["status"] == ref["status"] == 0
    dg = gpu["diag"]
    assert dg["admm_iterations"] == int(ref["sel_iters"].sum())
    # diagnostics: iteration histogram and the near-threshold count (margin
    # ||v_i| - lambda/rho| <= 1e-6 of the final iterate, v = x + u) against the oracle's
    assert dg["admm_iter_hist"] == iteration_histogram(ref["sel_iters"], ref["sel_conv"])
    near = int(np.sum(np.abs(np.abs(ref["sel_v"]) - ref["lambdas"][None, :, None, None]) <= 1e-6))
    assert dg["admm_near_threshold"] == near
    assert dg["ms_support"] >= 0.0


def test_c1_device_pointers_match_host_pointers():
    d = synth.workload_data(1)
    kw = dict(B1=20, B2=10, q=16)
    host = native.uoi_fit_traced(d.X, d.y, **kw)
    Xd = torch.from_numpy(d.X).cuda()
    yd = torch.from_numpy(d.y).cuda().reshape(-1, 1)
    dev = native.uoi_fit_traced(Xd, yd, **kw)
    assert dev["beta"].is_cuda
    np.testing.assert_array_equal(dev["beta"].cpu().numpy(), host["beta"])
    np.testing.assert_array_equal(dev["sel_beta"].cpu().numpy(), host["sel_beta"])


def test_c1_cold_start_and_mean_bagging():
    d = synth.workload_data(1)
    kw = dict(B1=6, B2=5, q=10, warm_start=0, bagging=1, split_mode=1, seed=7, problem_id=3)
    ref = oracle.uoi_lasso_fit(d.X, d.y, B1=6, B2=5, q=10, warm_start=0, bagging=1,
                               split_fixed=1, seed=7, problem_id=3)
    gpu = native.uoi_fit_traced(d.X, d.y, **kw)
    compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), block_len=0, seed=7, problem_id=3,
                split_mode=1)


@pytest.mark.parametrize("n,p,nnz", [(203, 77, 8), (64, 1, 1), (300, 128, 12)])
def test_ragged_sizes_resident(n, p, nnz):
    d = synth.lasso_problem(n, p, nnz, seed=n + p, sigma=0.5)
    kw = dict(B1=5, B2=4, q=7)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, **kw)
    compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), **kw)


@pytest.mark.parametrize("warm", [1, 0])
def test_streaming_schedule_fp64(warm):
    # p > 128 in FP64 takes the per-iteration (streaming) schedule: GEMV for the
    # single path chain per bootstrap, tiled GEMM for the cold lambda batch.
    d = synth.lasso_problem(420, 150, 15, seed=11, sigma=0.5)
    kw = dict(B1=3, B2=3, q=6, warm_start=warm)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, **kw)
    compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), **kw)


def test_var_small_fp64_parity():
    vp = synth.var_problem(24, 400, 0.1, 0.8, seed=5, burn_in=100)
    kw = dict(B1=6, B2=5, q=8, block_len=25)
    ref = oracle.uoi_var_fit(vp.series, **kw)
    S = vp.series
    gpu = native.uoi_fit_traced(S[:-1], S[1:], **kw)
    compare_fit(ref, gpu, S[:-1], S[1:], **kw)
    out = native.uoi_var_fit(S, **kw)
    np.testing.assert_array_equal(out["A"][0], gpu["beta"])
    assert np.all(out["mu"] == 0)


def test_var_streaming_gemm_fp64():
    vp = synth.var_problem(140, 500, 0.03, 0.8, seed=6, burn_in=100)
    kw = dict(B1=3, B2=3, q=5, block_len=40)
    ref = oracle.uoi_var_fit(vp.series, **kw)
    S = vp.series
    gpu = native.uoi_fit_traced(S[:-1], S[1:], **kw)
    compare_fit(ref, gpu, S[:-1], S[1:], **kw)


@pytest.mark.parametrize("warm", [0, 1])
def test_lasso_admm_batch_parity(warm):
    d = synth.workload_data(1)
    n = d.X.shape[0]
    w = np.stack([oracle.selection_weights(n, 0, 0, 0, k) for k in range(5)])
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 12)
    ref = oracle.lasso_admm_batch(d.X, d.y, w, lam, warm_start=warm)
    gpu = native.lasso_admm_batch(d.X, d.y, w, lam, warm_start=warm)
    np.testing.assert_array_equal(gpu["iters"], ref["iters"])
    for idx in np.ndindex(*ref["beta"].shape[:3]):
        assert rel_l2(gpu["beta"][idx], ref["beta"][idx]) <= 1e-6
    assert np.array_equal(gpu["beta"] != 0, ref["beta"] != 0)


def test_edge_cases_single_bootstrap_and_lambda():
    d = synth.workload_data(1)
    kw = dict(B1=1, B2=1, q=1)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, **kw)
    compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), **kw)


def test_lambda_above_max_gives_empty_family_and_zero_beta():
    d = synth.workload_data(1)
    lmax = oracle.lambda_max(d.X, d.y)
    lam = np.array([2.0 * lmax, 1.5 * lmax])
    gpu = native.uoi_fit_traced(d.X, d.y, B1=4, B2=3, q=2, lambdas=lam)
    assert np.all(gpu["family"] == 0)
    assert np.all(gpu["beta"] == 0)
    # loss of the empty model is the held-out sum of squares
    for k in range(3):
        ev = gpu["est_eval"][k].astype(bool)
        np.testing.assert_allclose(gpu["est_loss"][k, :, 0], np.sum(d.y[ev] ** 2), rtol=1e-12)


def test_max_iter_one_warns_and_nan_rejected():
    d = synth.workload_data(1)
    out = native.uoi_fit_traced(d.X, d.y, B1=2, B2=2, q=3, max_iter=1)
    assert out["status"] == native.OK_WITH_WARNINGS
    assert np.all(out["sel_iters"] == 1)
    assert out["diag"]["admm_nonconverged"] > 0
    assert out["diag"]["admm_iter_hist"] == iteration_histogram(out["sel_iters"], out["sel_conv"])
    assert out["diag"]["admm_iter_hist"][7] == out["diag"]["admm_nonconverged"]
    Xn = d.X.copy()
    Xn[5, 7] = np.inf
    with pytest.raises(native.UoiError) as ei:
        native.uoi_fit_traced(Xn, d.y, B1=2, B2=2, q=3)
    assert ei.value.status == native.ERR_NONFINITE


def test_mixed_form_c1_within_1e5():
    d = synth.workload_data(1)
    kw = dict(B1=20, B2=10, q=16)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, precision=native.PREC_MIXED, **kw)
    assert gpu["diag"]["admm_iter_hist"] == iteration_histogram(gpu["sel_iters"], gpu["sel_conv"])
    fam_g = bits_to_bool(gpu["family"], 50)
    fam_r = bits_to_bool(ref["family"], 50)
    assert (fam_g != fam_r).sum() == 0
    assert rel_l2(gpu["beta"], ref["beta"]) <= 1e-5


@pytest.mark.parametrize("warm", [0, 1])
def test_mixed_tensor_core_xupdate_vs_oracle(warm):
    # p > 192 in the mixed form takes the tensor-core x-update (two-piece fp16 split,
    # three products, compensated accumulation); every column must meet the stopping
    # rule in exact arithmetic up to the mixed form's rounding, sit within its KKT
    # residual / lambda_min(H) of the exact minimiser, and share its support outside
    # the band that residual leaves open (mixed_check).
    d = synth.lasso_problem(1200, 300, 20, seed=31, sigma=0.5, toeplitz_rho=0.5)
    n = d.X.shape[0]
    w = np.stack([oracle.selection_weights(n, 0, 0, 0, k) for k in range(3)])
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 8)
    ref = oracle.lasso_admm_batch(d.X, d.y, w, lam, warm_start=warm)
    gpu = native.lasso_admm_batch(d.X, d.y, w, lam, warm_start=warm, precision=native.PREC_MIXED)
    assert gpu["conv"].all()
    rep = mixed_check.check_batch(d.X, d.y, w, lam, gpu["beta"], ref["beta"], mixed_check.ETA_MIXED)
    print(rep)
    assert np.abs(gpu["iters"].astype(int) - ref["iters"]).max() <= max(3, int(0.1 * ref["iters"].max()))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ols_duplicate_column_goes_to_fp64_factor(prec):
    # With an exact duplicate column every support holding both copies is singular:
    # the FP32-factor solver must refuse it (pivot far below 1e-3 of the largest
    # diagonal) and hand it to the FP64 factor, which flags it and solves it by the
    # ADMM at lambda = 0 (the minimum-norm solution: the pair shares the weight).
    # Supports without the pair stay on the refined FP32 factor and agree with the
    # oracle's FP64 Cholesky to FP64 rounding (FP64 form).
    d = synth.lasso_problem(500, 20, 6, seed=21, sigma=0.5)
    X = d.X.copy()
    X[:, 1] = X[:, 0]
    kw = dict(B1=4, B2=3, q=10)
    precision = native.PREC_FP64 if prec == "fp64" else native.PREC_MIXED
    gpu = native.uoi_fit_traced(X, d.y, precision=precision, **kw)
    fam = bits_to_bool(gpu["family"], 20)[:, 0, :]
    pair = fam[:, 0] & fam[:, 1]
    assert pair.any()
    assert gpu["diag"]["ols_fp64"] > 0
    assert np.isfinite(gpu["est_loss"]).all() and np.isfinite(gpu["beta"]).all()
    if prec == "fp64":
        # exact FP64 moments: the pair's pivot is at rounding level, below 1e-12
        # (the mixed form's FP32-accurate Gram leaves a ~1e-7 pivot instead)
        assert gpu["status"] == native.OK_WITH_WARNINGS
        sing = gpu["est_singular"][:, :, 0].astype(bool)
        np.testing.assert_array_equal(sing, np.broadcast_to(pair, sing.shape))
        ref = oracle.uoi_lasso_fit(X, d.y, **kw)
        assert np.array_equal(bits_to_bool(ref["family"], 20), bits_to_bool(gpu["family"], 20))
        # every loss (singular supports included: the duplicates agree on every row)
        np.testing.assert_allclose(gpu["est_loss"], ref["est_loss"], rtol=1e-9, atol=1e-12)
        np.testing.assert_array_equal(gpu["est_jstar"], ref["est_jstar"])
        # chosen estimates, singular or not, against the oracle's minimum-norm solutions
        for k in range(3):
            want = ref["est_beta"][k, ref["est_jstar"][k], 0]
            assert rel_l2(gpu["est_beta"][k, 0], want) <= 1e-9
            if pair[ref["est_jstar"][k]]:
                assert abs(gpu["est_beta"][k, 0, 0] - gpu["est_beta"][k, 0, 1]) <= 1e-8 * abs(want[0])
        assert rel_l2(gpu["beta"], ref["beta"]) <= 1e-9


def test_mixed_tensor_core_inverse_vs_oracle():
    # p >= 512 in the mixed form inverts G/n + rho I by the block Schur-complement
    # recursion on FP32-accurate tensor-core GEMMs (p = 700 recurses twice, with
    # ragged 316- and 60-order blocks); held to the exact minimiser as above.
    d = synth.lasso_problem(2500, 700, 40, seed=33, sigma=0.5, toeplitz_rho=0.5)
    n = d.X.shape[0]
    w = np.stack([oracle.selection_weights(n, 0, 0, 0, k) for k in range(3)])
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 8)
    ref = oracle.lasso_admm_batch(d.X, d.y, w, lam, warm_start=0)
    gpu = native.lasso_admm_batch(d.X, d.y, w, lam, warm_start=0, precision=native.PREC_MIXED)
    assert gpu["conv"].all()
    rep = mixed_check.check_batch(d.X, d.y, w, lam, gpu["beta"], ref["beta"], mixed_check.ETA_MIXED)
    print(rep)
    assert np.abs(gpu["iters"].astype(int) - ref["iters"]).max() <= max(3, int(0.1 * ref["iters"].max()))


def test_mixed_tensor_core_xupdate_many_chain_tiles():
    # r = 40 responses x 4 lambdas = 160 chains per bootstrap group: the
    # tensor-core x-update runs 3 chain tiles of <= 64 per group (the VAR layout)
    d = synth.lasso_problem(1500, 300, 20, seed=41, sigma=0.5, toeplitz_rho=0.5)
    g = np.random.Generator(np.random.PCG64(42))
    B = g.standard_normal((300, 40)) * (g.random((300, 40)) < 0.05)
    Y = d.X @ B + 0.5 * g.standard_normal((1500, 40))
    n = d.X.shape[0]
    w = np.stack([oracle.selection_weights(n, 0, 0, 0, k) for k in range(2)])
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, Y), 4)
    ref = oracle.lasso_admm_batch(d.X, Y, w, lam, warm_start=0)
    gpu = native.lasso_admm_batch(d.X, Y, w, lam, warm_start=0, precision=native.PREC_MIXED)
    assert gpu["conv"].all()
    rep = mixed_check.check_batch(d.X, Y, w, lam, gpu["beta"], ref["beta"], mixed_check.ETA_MIXED)
    print(rep)


def test_large_supports_factor_outside_shared_memory():
    # Two selection bootstraps and a small lambda_min leave supports of ~390
    # features: beyond the shared-memory factor of the refined OLS (~330), so the
    # factor lives in global scratch.  Plain form: losses and the fit as the oracle.
    d = synth.lasso_problem(4000, 400, 60, seed=43, sigma=0.5)
    kw = dict(B1=2, B2=2, q=5, lambda_min_ratio=1e-4)
    ref = oracle.uoi_lasso_fit(d.X, d.y, **kw)
    gpu = native.uoi_fit_traced(d.X, d.y, precision=native.PREC_FP64, **kw)
    fam = bits_to_bool(gpu["family"], 400)[:, 0, :]
    assert fam.sum(axis=1).max() > 330
    compare_fit(ref, gpu, d.X, d.y.reshape(-1, 1), **kw)
