"""Pins of the oracle's VAR(d) lagged design and unpenalised intercept against
facts fixed outside the oracle: exact noiseless VAR(d) recursions, sklearn's
coordinate-descent LASSO with a fitted intercept, numpy's least squares on
[X_S 1], shift invariance of the centred problem, and the lambda_max identity
of the centred data (Alg. 2, Eq. 6-9)."""
import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import synth


def _noiseless_var(p, d, T, seed, mu_scale=0.0, radius=0.95):
    """s_t = mu + sum_j A_j s_{t-j} exactly; the companion matrix has spectral
    radius ``radius`` and distinct complex eigenvalues."""
    g = np.random.Generator(np.random.PCG64(seed))
    A = g.uniform(0.2, 0.6, (d, p, p)) * g.choice([-1.0, 1.0], (d, p, p))
    comp = np.zeros((d * p, d * p))
    comp[:p] = np.concatenate(list(A), axis=1)
    comp[p:, :-p] = np.eye((d - 1) * p)
    A *= radius / np.max(np.abs(np.linalg.eigvals(comp)))
    mu = mu_scale * g.standard_normal(p)
    S = np.zeros((T, p))
    S[:d] = 3.0 * g.standard_normal((d, p))
    for t in range(d, T):
        S[t] = mu + sum(A[j] @ S[t - 1 - j] for j in range(d))
    return S, A, mu


@pytest.mark.parametrize("d", [1, 2, 3])
def test_lagged_design_reproduces_var_recursion(d):
    S, A, _ = _noiseless_var(4, d, 40, seed=30 + d)
    X, Y = oracle.lagged_design(S, d)
    assert X.shape == (40 - d, 4 * d) and Y.shape == (40 - d, 4)
    # Eq. 6-8: Y = X B with B^T = (A_1 ... A_d)
    np.testing.assert_allclose(Y, X @ np.concatenate(list(A), axis=1).T, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(Y, S[d:])


def test_lagged_design_order_one_is_the_pairing_of_successive_rows():
    S = synth.var_problem(6, 50, 0.3, 0.8, seed=3, burn_in=10).series
    X, Y = oracle.lagged_design(S, 1)
    np.testing.assert_array_equal(X, S[:-1])
    np.testing.assert_array_equal(Y, S[1:])


def _offset_problem(seed, n=160, p=12):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, p)) + g.uniform(-4, 4, p)          # columns far from zero mean
    beta = np.zeros(p)
    beta[[1, 4, 9]] = [2.0, -1.5, 1.0]
    y = 5.0 + X @ beta + 0.3 * g.standard_normal(n)
    return X, y


def _centred_lambda_max(X, Y, w=None):
    w = np.ones(X.shape[0]) if w is None else np.asarray(w, dtype=float)
    Xc = X - (w @ X) / w.sum()
    Yc = Y - (w @ Y) / w.sum()
    return np.max(np.abs(Xc.T @ (w[:, None] * Yc))) / w.sum()


def test_lasso_intercept_against_sklearn():
    sk = pytest.importorskip("sklearn.linear_model")
    X, y = _offset_problem(1)
    n = X.shape[0]
    w = oracle.selection_weights(n, 0, 0, 0, 2)
    lam = oracle.lambda_grid(_centred_lambda_max(X, y[:, None], w), 12)
    out = oracle.lasso_admm_intercept(X, y, w, lam, abs_tol=1e-10, rel_tol=1e-10, max_iter=20000)
    assert out["status"] == 0
    Xr = np.repeat(X, w, axis=0)
    yr = np.repeat(y, w)
    for j in [1, 4, 8, 11]:
        m = sk.Lasso(alpha=lam[j], fit_intercept=True, tol=1e-13, max_iter=200000)
        m.fit(Xr, yr)
        np.testing.assert_allclose(out["beta"][j, 0], m.coef_, atol=1e-6)
        np.testing.assert_allclose(out["mu"][j, 0], m.intercept_, atol=1e-5)


def test_lasso_intercept_zero_above_centred_lambda_max():
    X, y = _offset_problem(2)
    n = X.shape[0]
    w = oracle.selection_weights(n, 0, 4, 0, 0)
    lmax = _centred_lambda_max(X, y[:, None], w)
    out = oracle.lasso_admm_intercept(X, y, w, np.array([lmax * 1.0001, lmax * 2.0]))
    assert np.all(out["beta"] == 0.0)
    np.testing.assert_allclose(out["mu"][:, 0], (w @ y) / w.sum(), rtol=1e-13)
    # just below lambda_max a coefficient is active
    below = oracle.lasso_admm_intercept(X, y, w, np.array([lmax * 0.98]), abs_tol=1e-9, rel_tol=1e-9,
                                        max_iter=5000)
    assert np.count_nonzero(below["beta"]) >= 1


def test_lasso_intercept_shift_invariance():
    X, y = _offset_problem(3)
    n, p = X.shape
    w = oracle.selection_weights(n, 0, 5, 0, 1)
    lam = oracle.lambda_grid(_centred_lambda_max(X, y[:, None], w), 6)
    a = oracle.lasso_admm_intercept(X, y, w, lam, abs_tol=1e-10, rel_tol=1e-10, max_iter=20000)
    cx = np.linspace(-7, 11, p)
    b = oracle.lasso_admm_intercept(X + cx, y - 3.0, w, lam, abs_tol=1e-10, rel_tol=1e-10,
                                    max_iter=20000)
    np.testing.assert_allclose(b["beta"], a["beta"], atol=1e-9)
    # y - 3 = (mu - 3 - cx^T beta) + (x + cx)^T beta
    shift = -3.0 - np.einsum("i,jei->je", cx, a["beta"])
    np.testing.assert_allclose(b["mu"], a["mu"] + shift, atol=1e-8)


def test_lasso_intercept_is_uncentred_lasso_on_centred_data():
    # data already centred under w: the intercept is zero and beta is the plain LASSO
    X, y = _offset_problem(4)
    n = X.shape[0]
    w = oracle.selection_weights(n, 0, 6, 0, 0)
    X = X - (w @ X) / w.sum()
    y = y - (w @ y) / w.sum()
    lam = oracle.lambda_grid(oracle.lambda_max(X, y), 5)
    a = oracle.lasso_admm_intercept(X, y, w, lam)
    b = oracle.lasso_admm_batch(X, y, w[None, :], lam)
    np.testing.assert_allclose(a["beta"], b["beta"][0], atol=1e-12)
    assert np.max(np.abs(a["mu"])) < 1e-12


def test_fit_intercept_ols_against_lstsq():
    X, y = _offset_problem(5, n=200, p=10)
    m, p = X.shape
    out = oracle.uoi_lasso_fit(X, y, 4, 3, 6, intercept=1)
    assert out["status"] in (0, 1)
    assert out["beta"].shape == (1, p + 1)
    fam = out["family"]
    for k in range(3):
        wt, ev = oracle.estimation_weights(m, 0, 0.8, 0, 0, 0, k)[:2]
        for j in range(6):
            S = [i for i in range(p) if int(fam[j, 0, i // 64]) >> (i % 64) & 1]
            D = np.concatenate([X[:, S], np.ones((m, 1))], axis=1)
            ref = np.linalg.lstsq(np.repeat(D, wt, axis=0), np.repeat(y, wt), rcond=None)[0]
            got = out["est_beta"][k, j, 0]
            np.testing.assert_allclose(got[S], ref[:-1], rtol=1e-9, atol=1e-10)
            np.testing.assert_allclose(got[p], ref[-1], rtol=1e-9, atol=1e-10)
            assert np.all(np.delete(got, S + [p]) == 0)
            # held-out loss: explicit residuals with the intercept
            res = (y - D @ ref)[ev.astype(bool)]
            np.testing.assert_allclose(out["est_loss"][k, j, 0], res @ res, rtol=1e-8)


def test_fit_intercept_lambda_max_from_centred_data():
    X, y = _offset_problem(6)
    out = oracle.uoi_lasso_fit(X, y, 2, 2, 4, intercept=1)
    np.testing.assert_allclose(out["lambdas"][0], _centred_lambda_max(X, y[:, None]), rtol=1e-12)


def test_fit_intercept_selection_shift_invariance():
    X, y = _offset_problem(7)
    kw = dict(B1=4, B2=3, q=8, intercept=1)
    a = oracle.uoi_lasso_fit(X, y, **kw)
    b = oracle.uoi_lasso_fit(X + 2.5, y + 10.0, **kw)
    np.testing.assert_array_equal(a["family"], b["family"])
    np.testing.assert_allclose(b["beta"][0, :-1], a["beta"][0, :-1], atol=1e-9)
    np.testing.assert_allclose(b["est_beta"][..., :-1], a["est_beta"][..., :-1], atol=1e-9)
    # per bootstrap and support: mu' = mu + 10 - 2.5 * sum(beta)
    shift = 10.0 - 2.5 * a["est_beta"][..., :-1].sum(axis=-1)
    np.testing.assert_allclose(b["est_beta"][..., -1], a["est_beta"][..., -1] + shift, atol=1e-8)


def _oscillating_var(p, d, T, seed, mu_scale=2.0):
    """Noiseless VAR(d) with intercept whose companion eigenvalues all lie on
    the unit circle (distinct angles), so the orbit keeps exciting every
    direction and the lagged design stays well conditioned.
    d = 1: A_1 = Q R Q^T with R 2 x 2 rotations (p even).
    d = 2: A_1 = Q diag(2 cos theta) Q^T, A_2 = -I: per mode the roots of
    z^2 - 2 cos(theta) z + 1, i.e. exp(+-i theta)."""
    g = np.random.Generator(np.random.PCG64(seed))
    Q = np.linalg.qr(g.standard_normal((p, p)))[0]
    theta = np.linspace(0.5, 2.5, p) + g.uniform(-0.1, 0.1, p)
    if d == 1:
        R = np.zeros((p, p))
        for i in range(0, p, 2):
            c, s = np.cos(theta[i]), np.sin(theta[i])
            R[i:i + 2, i:i + 2] = [[c, -s], [s, c]]
        A = np.stack([Q @ R @ Q.T])
    else:
        A = np.stack([Q @ np.diag(2 * np.cos(theta)) @ Q.T, -np.eye(p)])
    mu = mu_scale * g.standard_normal(p)
    S = np.zeros((T, p))
    S[:d] = 3.0 * g.standard_normal((d, p))
    for t in range(d, T):
        S[t] = mu + sum(A[j] @ S[t - 1 - j] for j in range(d))
    return S, A, mu


@pytest.mark.parametrize("d,p", [(1, 4), (2, 3)])
def test_var_fit_noiseless_recovery_with_intercept(d, p):
    # noiseless data, every true coefficient well above the smallest lambda:
    # the family holds the true support, whose OLS (with mu) is exact
    S, A, mu = _oscillating_var(p, d, 70, seed=0)
    out = oracle.uoi_var_fit(S, 5, 4, 10, order=d, intercept=1, block_len=6)
    assert out["status"] in (0, 1)
    np.testing.assert_allclose(out["A"], A, atol=1e-10)
    np.testing.assert_allclose(out["mu"], mu, atol=1e-10)
    Ac, muc, st = oracle.uoi_var_fit_c(S, 5, 4, 10, order=d, intercept=1, block_len=6)
    assert st == out["status"]
    np.testing.assert_array_equal(Ac, out["A"])
    np.testing.assert_array_equal(muc, out["mu"])


def test_var_fit_order_two_without_intercept_partition():
    vp = synth.var_problem(4, 150, 0.4, 0.7, seed=11, burn_in=40)
    out = oracle.uoi_var_fit(vp.series, 3, 3, 5, order=2, block_len=10)
    p = 4
    # beta row e = (A_1[e, :], A_2[e, :])
    for j in range(2):
        np.testing.assert_array_equal(out["A"][j], out["beta"][:, j * p:(j + 1) * p])
    assert np.all(out["mu"] == 0)
    Ac, muc, st = oracle.uoi_var_fit_c(vp.series, 3, 3, 5, order=2, block_len=10)
    np.testing.assert_array_equal(Ac, out["A"])
    assert np.all(muc == 0)


def test_var_fit_argument_errors():
    S = np.zeros((5, 3))
    assert oracle.uoi_var_fit_c(S, 2, 2, 2, order=0)[2] == oracle.ERR_INVALID_ARG
    assert oracle.uoi_var_fit_c(S, 2, 2, 2, order=4)[2] == oracle.ERR_INVALID_ARG


def test_scalar_ar2_with_intercept_noiseless_recovery():
    # p = 1, d = 2: s_t = mu + 2 cos(theta) s_{t-1} - s_{t-2}, roots exp(+-i theta)
    theta, mu = 0.9, 1.5
    S = np.zeros((60, 1))
    S[0, 0], S[1, 0] = 2.0, -1.0
    for t in range(2, 60):
        S[t, 0] = mu + 2 * np.cos(theta) * S[t - 1, 0] - S[t - 2, 0]
    out = oracle.uoi_var_fit(S, 4, 3, 8, order=2, intercept=1, block_len=4)
    np.testing.assert_allclose(out["A"][:, 0, 0], [2 * np.cos(theta), -1.0], atol=1e-10)
    np.testing.assert_allclose(out["mu"], [mu], atol=1e-10)
