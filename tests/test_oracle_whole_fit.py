"""Pins of the oracle's whole UoI fit (Alg. 1, Alg. 2).  The general case, with
real selection, is at the end of this file.  First the cases where the selection
step is decided in advance, so that the estimation step has an independent
route: at an explicit lambda far below every |Xᵀy|/n the LASSO keeps every
feature in every bootstrap (the intersection, Eq. 3, is the full set); at a
lambda above lambda_max it keeps none.  Then each estimation bootstrap's
coefficients are the least-squares fit on its training draws (numpy lstsq on
the rows scaled by sqrt(w), not the oracle's Cholesky), its held-out loss is the
sum of squared residuals on the evaluation rows (the traced loss: the 1/|E|
factor does not change the argmin), j* is the argmin, and beta* the
median (or mean) over bootstraps.  For VAR(d) (Alg. 2) the same holds per
equation on the lagged design of Eq. 7-8 (built here with numpy), with block
bootstrap draws and, with an intercept, a ones column whose coefficient is mu.
The bootstrap and split weights come from the oracle's Philox functions,
pinned separately by known-answer vectors.
"""
import numpy as np
import pytest

import oracle

SEED = 5


def _problem(n=300, p=6, seed=3):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, p))
    beta = g.uniform(0.5, 2.0, size=p) * g.choice([-1.0, 1.0], size=p)
    y = X @ beta + 0.3 * g.standard_normal(n)
    return X, y


def _train_eval(m, B2, split_fixed=0):
    out = []
    for k in range(B2):
        w, ev, _ = oracle.estimation_weights(m, 0, 0.8, split_fixed, SEED, 0, k)
        out.append((w.astype(np.float64), ev.astype(bool)))
    return out


def _wls(X, y, w):
    sw = np.sqrt(w)
    return np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)[0]


@pytest.mark.parametrize("bagging,split_fixed", [(0, 0), (1, 0), (0, 1)])   # median / mean; per-bootstrap / fixed split
def test_dense_support_reduces_to_least_squares_on_the_training_draws(bagging, split_fixed):
    X, y = _problem()
    n, p = X.shape
    B1, B2 = 4, 3
    fit = oracle.uoi_lasso_fit(X, y, B1, B2, 1, lambdas=np.array([1e-9]), bagging=bagging, seed=SEED,
                               max_iter=5000, split_fixed=split_fixed)
    assert fit["status"] >= 0
    # every selection bootstrap keeps every feature: the family is the full set
    assert np.all(fit["sel_beta"] != 0.0)
    assert int(fit["family"][0, 0, 0]) == (1 << p) - 1
    splits = _train_eval(n, B2, split_fixed)
    if split_fixed:                                   # one evaluation set for every bootstrap
        assert all(np.array_equal(splits[0][1], ev) for _, ev in splits)
    ests = np.stack([_wls(X, y, w) for w, _ in splits])
    np.testing.assert_allclose(fit["est_beta"][:, 0, 0, :], ests, rtol=1e-9, atol=1e-12)
    want = np.median(ests, axis=0) if bagging == 0 else np.mean(ests, axis=0)
    np.testing.assert_allclose(fit["beta"][0], want, rtol=1e-9, atol=1e-12)


def test_argmin_takes_the_full_support_over_the_empty_one():
    X, y = _problem(seed=4)
    n, p = X.shape
    B1, B2 = 3, 4
    lmax = np.max(np.abs(X.T @ y)) / n
    lambdas = np.array([100.0 * lmax, 1e-9])          # descending: empty support, then all
    fit = oracle.uoi_lasso_fit(X, y, B1, B2, 2, lambdas=lambdas, seed=SEED, max_iter=5000)
    assert fit["status"] >= 0
    assert np.all(fit["sel_beta"][:, 0] == 0.0) and np.all(fit["sel_beta"][:, 1] != 0.0)
    assert int(fit["family"][0, 0, 0]) == 0 and int(fit["family"][1, 0, 0]) == (1 << p) - 1
    ests = []
    for k, (w, ev) in enumerate(_train_eval(n, B2)):
        b = _wls(X, y, w)
        loss_empty = np.sum(y[ev] ** 2)
        loss_full = np.sum((y[ev] - X[ev] @ b) ** 2)
        np.testing.assert_allclose(fit["est_loss"][k, 0, 0], loss_empty, rtol=1e-12)
        np.testing.assert_allclose(fit["est_loss"][k, 1, 0], loss_full, rtol=1e-8)
        assert loss_full < loss_empty
        assert fit["est_jstar"][k] == 1
        ests.append(b)
    np.testing.assert_allclose(fit["beta"][0], np.median(np.stack(ests), axis=0), rtol=1e-9, atol=1e-12)


def _lagged(S, order):
    """Eq. 7-8 written out: row t holds X_{t-1}, ..., X_{t-order} (lag 1 first), response X_t."""
    N = S.shape[0]
    X = np.hstack([S[order - j:N - j] for j in range(1, order + 1)])
    return X, S[order:]


@pytest.mark.parametrize("order,intercept", [(1, 0), (2, 1)])
def test_var_dense_support_reduces_to_per_equation_least_squares(order, intercept):
    # Alg. 2 with every lag kept in every bootstrap: each equation's estimate is the
    # least-squares fit on the block-bootstrap training draws of the lagged design
    g = np.random.Generator(np.random.PCG64(9))
    p, N = 4, 420
    A_true = 0.3 * g.standard_normal((order, p, p))
    S = np.zeros((N, p))
    for t in range(N):
        S[t] = 0.5 + g.standard_normal(p)
        for j in range(1, min(order, t) + 1):
            S[t] += A_true[j - 1] @ S[t - j]
    B1, B2, L = 3, 3, 20
    fit = oracle.uoi_var_fit(S, B1, B2, 1, order=order, lambdas=np.array([1e-9]), block_len=L, seed=SEED,
                             intercept=intercept, max_iter=5000)
    assert fit["status"] >= 0
    X, Y = _lagged(S, order)
    m = X.shape[0]
    Z = np.hstack([X, np.ones((m, 1))]) if intercept else X
    ests = []
    for k in range(B2):
        w, _, _ = oracle.estimation_weights(m, L, 0.8, 0, SEED, 0, k)
        sw = np.sqrt(w.astype(np.float64))
        ests.append(np.linalg.lstsq(Z * sw[:, None], Y * sw[:, None], rcond=None)[0].T)   # (p, cols)
    want = np.median(np.stack(ests), axis=0)
    A_want = want[:, :order * p].reshape(p, order, p).transpose(1, 0, 2)
    np.testing.assert_allclose(fit["A"], A_want, rtol=1e-8, atol=1e-10)
    if intercept:
        np.testing.assert_allclose(fit["mu"], want[:, order * p], rtol=1e-8, atol=1e-10)


# ---- the general case: selection by an independent LASSO solver --------------------
# With real selection (supports that vary with lambda and bootstrap) the whole fit has
# an independent route too: each selection bootstrap's LASSO (Eq. 1, the weighted
# least squares over n_k = sum(w) draws plus lambda ||beta||_1) solved by
# scikit-learn's coordinate descent on the bootstrap's rows repeated by multiplicity;
# supports, their intersection (Eq. 3), least squares on each estimation bootstrap's
# training draws, held-out losses, argmin and the median by numpy.  The fixtures are
# chosen so that the comparison is decided: every active coefficient is far from
# zero and every inactive feature's correlation far from lambda, relative to the
# solvers' errors, and the two smallest distinct losses of each estimation bootstrap
# are apart.  Both margins are asserted.


def _sk_lasso(Xk, yk, lam, intercept=False):
    lm = pytest.importorskip("sklearn.linear_model")
    b = lm.Lasso(alpha=lam, fit_intercept=intercept, tol=1e-14, max_iter=10**6).fit(Xk, yk).coef_
    if intercept:                                              # the unpenalised mean, eliminated
        Xk, yk = Xk - Xk.mean(axis=0), yk - yk.mean()
    grad = Xk.T @ (yk - Xk @ b) / Xk.shape[0]
    act = b != 0
    assert np.all(np.abs(b[act]) > 1e-5)                       # active: clear of zero
    assert np.all(np.abs(grad[~act]) < lam * (1 - 1e-4))       # inactive: clear of lambda
    return b


def _independent_uoi(X, Y, lambdas, B1, B2, block_len, intercept=False):
    """Alg. 1 per response column of Y, every step outside the oracle; with an
    intercept, estimates carry the unpenalised mean as their last entry."""
    m, p = X.shape
    q, r = len(lambdas), Y.shape[1]
    pa = p + (1 if intercept else 0)
    fam = np.ones((q, r, p), dtype=bool)
    for k in range(B1):
        rows = np.repeat(np.arange(m), oracle.selection_weights(m, block_len, SEED, 0, k).astype(np.int64))
        for e in range(r):
            for j, lam in enumerate(lambdas):
                fam[j, e] &= _sk_lasso(X[rows], Y[rows, e], lam, intercept) != 0
    chosen = np.zeros((B2, r, pa))
    jstar = np.zeros(B2, dtype=int)
    for k in range(B2):
        w, ev, _ = oracle.estimation_weights(m, block_len, 0.8, 0, SEED, 0, k)
        sw, ev = np.sqrt(w.astype(np.float64)), ev.astype(bool)
        losses = np.zeros(q)
        ests = np.zeros((q, r, pa))
        for j in range(q):
            for e in range(r):
                cols = list(np.flatnonzero(fam[j, e])) + ([p] if intercept else [])
                Z = np.hstack([X, np.ones((m, 1))]) if intercept else X
                if cols:
                    ests[j, e, cols] = np.linalg.lstsq(Z[:, cols] * sw[:, None], Y[:, e] * sw, rcond=None)[0]
                losses[j] += np.sum((Y[ev, e] - Z[ev] @ ests[j, e]) ** 2)
        jstar[k] = int(np.argmin(losses))                      # first of equal losses
        distinct = np.unique(losses)
        if distinct.size > 1:
            assert distinct[1] - distinct[0] > 1e-9 * distinct[0]
        chosen[k] = ests[jstar[k]]
    return fam, jstar, np.median(chosen, axis=0)


def _family_bits(fam):
    q, r, p = fam.shape
    return np.array([[sum(1 << i for i in range(p) if fam[j, e, i]) for e in range(r)] for j in range(q)])


def test_general_lasso_fit_matches_an_independent_route():
    g = np.random.Generator(np.random.PCG64(21))
    n, p = 400, 10
    X = g.standard_normal((n, p))
    truth = np.zeros(p)
    truth[[0, 3, 7]] = [1.5, -1.0, 0.6]
    y = X @ truth + 0.5 * g.standard_normal(n)
    lmax = np.max(np.abs(X.T @ y)) / n
    lambdas = lmax * np.array([0.6, 0.3, 0.1, 0.03, 0.01])
    B1, B2 = 5, 4
    fit = oracle.uoi_lasso_fit(X, y, B1, B2, len(lambdas), lambdas=lambdas, seed=SEED, max_iter=100000,
                               abs_tol=1e-11, rel_tol=1e-11)
    assert fit["status"] == 0 and np.all(fit["sel_conv"] == 1)
    fam, jstar, beta = _independent_uoi(X, y[:, None], lambdas, B1, B2, 0)
    assert len({tuple(f) for f in fam[:, 0]}) >= 3              # the family really varies with lambda
    assert np.array_equal(fit["family"][:, :, 0].astype(np.int64), _family_bits(fam))
    assert np.array_equal(fit["est_jstar"], jstar)
    np.testing.assert_allclose(fit["beta"][0], beta[0], rtol=1e-9, atol=1e-12)


def test_general_lasso_fit_with_intercept_matches_an_independent_route():
    # the unpenalised intercept: selection with the means eliminated, estimation by
    # least squares on [X_S 1], mu the last entry of beta*
    g = np.random.Generator(np.random.PCG64(41))
    n, p = 400, 8
    X = g.standard_normal((n, p)) + 0.7
    truth = np.zeros(p)
    truth[[1, 4, 6]] = [1.2, -0.8, 0.5]
    y = 2.0 + X @ truth + 0.5 * g.standard_normal(n)
    Xc, yc = X - X.mean(axis=0), y - y.mean()
    lambdas = np.max(np.abs(Xc.T @ yc)) / n * np.array([0.6, 0.3, 0.1, 0.03])
    B1, B2 = 4, 3
    fit = oracle.uoi_lasso_fit(X, y, B1, B2, len(lambdas), lambdas=lambdas, seed=SEED, max_iter=100000,
                               abs_tol=1e-11, rel_tol=1e-11, intercept=1)
    assert fit["status"] == 0
    fam, jstar, beta = _independent_uoi(X, y[:, None], lambdas, B1, B2, 0, intercept=True)
    assert len({tuple(f) for f in fam[:, 0]}) >= 3
    assert np.array_equal(fit["family"][:, :, 0].astype(np.int64), _family_bits(fam))
    assert np.array_equal(fit["est_jstar"], jstar)
    np.testing.assert_allclose(fit["beta"][0], beta[0], rtol=1e-9, atol=1e-12)


def test_general_var_fit_matches_an_independent_route():
    # Alg. 2: p equations sharing the lagged design (Eq. 7-9), block bootstrap draws,
    # one lambda grid; j* is chosen once per estimation bootstrap over the summed
    # losses of all equations
    g = np.random.Generator(np.random.PCG64(33))
    p, N, L = 4, 500, 25
    A1 = np.diag([0.6, -0.5, 0.4, 0.3])
    A1[0, 2], A1[3, 1] = 0.35, -0.3
    S = np.zeros((N, p))
    for t in range(1, N):
        S[t] = A1 @ S[t - 1] + 0.5 * g.standard_normal(p)
    X, Y = _lagged(S, 1)
    lmax = np.max(np.abs(X.T @ Y)) / X.shape[0]
    lambdas = lmax * np.array([0.5, 0.2, 0.08, 0.03])
    B1, B2 = 4, 3
    fit = oracle.uoi_var_fit(S, B1, B2, len(lambdas), order=1, lambdas=lambdas, block_len=L, seed=SEED,
                             max_iter=100000, abs_tol=1e-11, rel_tol=1e-11)
    assert fit["status"] == 0
    fam, jstar, beta = _independent_uoi(X, Y, lambdas, B1, B2, L)
    assert len({fam[j].tobytes() for j in range(len(lambdas))}) >= 3
    assert np.array_equal(fit["family"][:, :, 0].astype(np.int64), _family_bits(fam))
    assert np.array_equal(fit["est_jstar"], jstar)
    np.testing.assert_allclose(fit["A"][0], beta, rtol=1e-9, atol=1e-12)
