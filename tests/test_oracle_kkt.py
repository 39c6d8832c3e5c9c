"""Pins of the oracle's exact LASSO minimiser (KKT polish) and its error bounds.

The polish is the reference of the error statements for forms that stop ADMM at
a tolerance (Eq. 5): it solves the active-set equation of the LASSO optimality
conditions (Eq. 2 with the 1/(2 n_k) scaling) and certifies the result.  Pinned
against brute-force enumeration of all sign patterns (p <= 8), the closed form
S_lambda(X^T y / n) for an orthonormal design, the empty solution above
lambda_max, scikit-learn's coordinate descent on replicated rows, and the
strong-convexity bounds that tie any point's KKT residual to its distance from
the minimiser.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import synth


def _moments(X, y, w=None):
    G, B = oracle.weighted_moments(X, y, w)
    nk = float(X.shape[0] if w is None else np.sum(w))
    return G, B[:, 0], nk


def _brute_force(G, b, nk, lam):
    """Exact minimiser by enumerating every sign pattern (3^p cases)."""
    p = G.shape[0]
    best = None
    for s in itertools.product((-1, 0, 1), repeat=p):
        s = np.array(s, dtype=float)
        A = np.flatnonzero(s)
        beta = np.zeros(p)
        if len(A):
            beta[A] = np.linalg.solve(G[np.ix_(A, A)], b[A] - nk * lam * s[A])
            if np.any(np.sign(beta[A]) != s[A]):
                continue
        grad = (b - G @ beta) / nk
        off = np.setdiff1d(np.arange(p), A)
        if np.all(np.abs(grad[off]) <= lam * (1 + 1e-12)):
            best = beta
    assert best is not None
    return best


def _problem(n, p, seed, w_k=None):
    g = np.random.Generator(np.random.PCG64(500 + seed))
    X = g.standard_normal((n, p))
    beta = np.zeros(p)
    beta[: max(1, p // 2)] = g.uniform(1, 2, max(1, p // 2)) * g.choice([-1, 1], max(1, p // 2))
    y = X @ beta + 0.5 * g.standard_normal(n)
    w = None if w_k is None else oracle.selection_weights(n, 0, 0, 0, w_k)
    return X, y, w


@pytest.mark.parametrize("p,seed", [(5, 0), (7, 1), (8, 2)])
def test_polish_of_admm_equals_brute_force(p, seed):
    X, y, w = _problem(40, p, seed, w_k=seed)
    G, b, nk = _moments(X, y, w)
    lam = oracle.lambda_grid(oracle.lambda_max(X, y), 6)
    out = oracle.lasso_admm_batch(X, y, w[None, :], lam, warm_start=1)
    for j in range(6):
        exact = _brute_force(G, b, nk, lam[j])
        pol = oracle.kkt_polish(G, b, nk, lam[j], out["beta"][0, j, 0])
        assert pol["certified"]
        np.testing.assert_allclose(pol["beta"], exact, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(pol["grad"], (b - G @ exact) / nk, rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("start", ["empty", "full", "wrong_signs"])
def test_polish_from_a_wrong_support_still_reaches_the_minimiser(start):
    X, y, w = _problem(60, 8, 7, w_k=3)
    G, b, nk = _moments(X, y, w)
    lam = 0.3 * oracle.lambda_max(X, y)
    exact = _brute_force(G, b, nk, lam)
    z0 = {"empty": np.zeros(8), "full": np.ones(8), "wrong_signs": -np.sign(exact) + (exact == 0)}[start]
    pol = oracle.kkt_polish(G, b, nk, lam, z0)
    assert pol["certified"] and pol["moves"] > 0
    np.testing.assert_allclose(pol["beta"], exact, rtol=1e-12, atol=1e-13)


def test_polish_orthonormal_closed_form():
    g = np.random.Generator(np.random.PCG64(3))
    n, p = 120, 12
    Q, _ = np.linalg.qr(g.standard_normal((n, p)))
    X = np.sqrt(n) * Q                                   # X^T X / n = I
    beta = np.zeros(p)
    beta[[1, 4, 7]] = [2.0, -1.5, 0.7]
    y = X @ beta + 0.3 * g.standard_normal(n)
    G, b, nk = _moments(X, y)
    c = X.T @ y / n
    for lam in [0.01, 0.1, 0.5, 1.0]:
        exact = np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)       # S_lambda(X^T y / n)
        pol = oracle.kkt_polish(G, b, nk, lam, np.zeros(p))
        assert pol["certified"]
        np.testing.assert_allclose(pol["beta"], exact, atol=1e-13)


def test_polish_is_zero_above_lambda_max():
    d = synth.workload_data(1)
    G, b, nk = _moments(d.X, d.y)
    lmax = oracle.lambda_max(d.X, d.y)
    pol = oracle.kkt_polish(G, b, nk, 1.0001 * lmax, np.ones(d.X.shape[1]))
    assert pol["certified"] and np.all(pol["beta"] == 0)
    pol = oracle.kkt_polish(G, b, nk, 0.999 * lmax, np.zeros(d.X.shape[1]))
    assert pol["certified"] and np.count_nonzero(pol["beta"]) == 1


def test_polish_against_sklearn_on_replicated_rows():
    sk = pytest.importorskip("sklearn.linear_model")
    d = synth.workload_data(1)
    n, p = d.X.shape
    w = oracle.selection_weights(n, 0, 0, 0, 1)
    G, b, nk = _moments(d.X, d.y, w)
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 16)
    out = oracle.lasso_admm_batch(d.X, d.y, w[None, :], lam)
    Xr = np.repeat(d.X, w, axis=0)
    yr = np.repeat(d.y, w)
    for j in [2, 6, 10, 15]:
        m = sk.Lasso(alpha=lam[j], fit_intercept=False, tol=1e-14, max_iter=1000000)
        m.fit(Xr, yr)
        pol = oracle.kkt_polish(G, b, nk, lam[j], out["beta"][0, j, 0])
        assert pol["certified"]
        np.testing.assert_allclose(pol["beta"], m.coef_, atol=1e-9)


def test_kkt_residual_is_zero_at_the_minimiser_and_exact_for_a_shift():
    X, y, w = _problem(80, 6, 11, w_k=5)
    G, b, nk = _moments(X, y, w)
    lam = 0.2 * oracle.lambda_max(X, y)
    exact = _brute_force(G, b, nk, lam)
    assert oracle.kkt_residual(G, b, nk, lam, exact) <= 1e-13
    # a point of the same support and signs moved by d: the residual is ||(H d)_A||
    # on the support plus the excess over lam off it
    A = exact != 0
    d = np.where(A, 1e-3 * np.arange(1, 7), 0.0)
    z = exact + d
    assert np.all(np.sign(z[A]) == np.sign(exact[A]))
    g = (b - G @ z) / nk
    want = np.concatenate([(g - lam * np.sign(z))[A], (np.abs(g) - np.minimum(np.abs(g), lam))[~A]])
    assert np.isclose(oracle.kkt_residual(G, b, nk, lam, z), np.linalg.norm(want), rtol=1e-12)


def test_admm_iterates_meet_the_stopping_bound_and_distance_bound():
    # every converged FP64 ADMM column: kkt_residual <= ||H|| eps_pri + eps_dual, and
    # its distance to the polished minimiser <= residual / lambda_min(H); supports
    # agree outside the band that residual leaves open
    d = synth.lasso_problem(300, 40, 8, seed=9, sigma=0.5, toeplitz_rho=0.5)
    n, p = d.X.shape
    w = np.stack([oracle.selection_weights(n, 0, 0, 0, k) for k in range(3)])
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 10)
    for warm in (0, 1):
        out = oracle.lasso_admm_batch(d.X, d.y, w, lam, warm_start=warm)
        assert out["conv"].all()
        for k in range(3):
            G, b, nk = _moments(d.X, d.y, w[k])
            H = G / nk
            ev = np.linalg.eigvalsh(H)
            mu, Hn = ev[0], ev[-1]
            for j in range(10):
                z = out["beta"][k, j, 0]
                kap = oracle.kkt_residual(G, b, nk, lam[j], z)
                assert kap <= oracle.admm_stop_bound(Hn, p, z, lam[j]) * (1 + 1e-9)
                pol = oracle.kkt_polish(G, b, nk, lam[j], z)
                assert pol["certified"]
                assert np.linalg.norm(z - pol["beta"]) <= kap / mu * (1 + 1e-9) + 1e-15
                band = oracle.support_band(pol["beta"], pol["grad"], lam[j], kap, mu, Hn)
                assert not (((z != 0) != (pol["beta"] != 0)) & ~band).any()


def test_support_band_catches_a_planted_wrong_sign_in_the_polish():
    # a polish that solved H_AA b_A = c_A + lam s_A (sign of the penalty flipped) would
    # not be certified and would disagree with brute force: the pin above then fails
    X, y, w = _problem(50, 6, 13, w_k=2)
    G, b, nk = _moments(X, y, w)
    lam = 0.3 * oracle.lambda_max(X, y)
    exact = _brute_force(G, b, nk, lam)
    A = np.flatnonzero(exact)
    wrong = np.zeros(6)
    wrong[A] = np.linalg.solve(G[np.ix_(A, A)], b[A] + nk * lam * np.sign(exact[A]))
    assert oracle.kkt_residual(G, b, nk, lam, wrong) > 1e-3
    assert np.max(np.abs(wrong - exact)) > 1e-3
