"""Pins of the FP64 oracle against facts outside itself (CPU only).

Each test ties one oracle function to something the paper or mathematics fixes:
published known-answer vectors, numpy's independent Philox, closed forms,
the KKT conditions of the LASSO (Eq. 2), lambda_max, brute-force enumeration
of supports, sklearn's coordinate-descent LASSO, numpy's min-norm least
squares, brute-force set logic for Eq. 3-4 and noiseless recovery.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Philox4x64-10 and the bootstrap index streams
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(h, 16) for h in row]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = oracle.philox4x64_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_matches_numpy():
    g = np.random.Generator(np.random.PCG64(7))
    for _ in range(50):
        ctr = [int(x) for x in g.integers(0, 2**63, size=4, dtype=np.uint64)]
        key = [int(x) for x in g.integers(0, 2**63, size=2, dtype=np.uint64)]
        # numpy's Philox adds one to the counter before producing its first block
        prev = list(ctr)
        prev[0] = (prev[0] - 1) % 2**64
        bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64),
                              key=np.array(key, dtype=np.uint64))
        want = [int(x) for x in bg.random_raw(4)]
        assert [int(x) for x in oracle.philox4x64_10(ctr, key)] == want


def _numpy_draws(seed, problem, k, tag, count):
    """Draw stream (k, tag) rebuilt from numpy's Philox and the documented layout."""
    out = []
    for blk in range((count + 3) // 4):
        # numpy increments its 256-bit counter (with carry) before the first
        # block, so start one below (blk, k, tag, 0)
        c = (blk | (k << 64) | (tag << 128)) - 1
        ctr = np.array([(c >> (64 * i)) % 2**64 for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(counter=ctr, key=np.array([seed, problem], dtype=np.uint64))
        out.extend(int(x) for x in bg.random_raw(4))
    return out[:count]


def test_draw_layout_matches_numpy():
    d = _numpy_draws(11, 3, 5, oracle.TAG_SELECTION, 10)
    for i in range(10):
        assert oracle.draw(11, 3, 5, oracle.TAG_SELECTION, i) == d[i]


def test_range_map_is_floor_of_product():
    g = np.random.Generator(np.random.PCG64(3))
    for _ in range(200):
        r = int(g.integers(0, 2**64 - 1, dtype=np.uint64))
        n = int(g.integers(1, 2**40))
        assert oracle.range_map(r, n) == (r * n) >> 64


@pytest.mark.parametrize("m,L", [(200, 0), (997, 1), (4999, 100), (19999, 200), (10, 10)])
def test_selection_weights_invariants(m, L):
    seed, prob = 0, 0
    for k in range(3):
        w = oracle.selection_weights(m, L, seed, prob, k)
        Lu = max(L, 1)
        units = (m + Lu - 1) // Lu
        # rebuild from numpy's Philox: units draws with replacement
        d = _numpy_draws(seed, prob, k, oracle.TAG_SELECTION, units)
        want = np.zeros(m, dtype=np.int64)
        for r in d:
            u = (r * units) >> 64
            want[u * Lu:min(u * Lu + Lu, m)] += 1
        np.testing.assert_array_equal(w, want)
        if Lu > 1:   # whole blocks only
            for b in range(units):
                blk = w[b * Lu:min(b * Lu + Lu, m)]
                assert np.all(blk == blk[0])
        else:
            assert int(w.sum()) == m


def test_selection_draws_chi_square():
    m = 64
    counts = np.zeros(m)
    for k in range(4000):
        counts += oracle.selection_weights(m, 0, 9, 0, k)
    exp = counts.sum() / m
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # 63 degrees of freedom: 99.9% quantile is ~103
    assert chi2 < 103.0


@pytest.mark.parametrize("m,L,fixed", [(200, 0, 0), (4999, 100, 0), (1001, 0, 1), (999, 50, 1)])
def test_estimation_split_invariants(m, L, fixed):
    Lu = max(L, 1)
    units = (m + Lu - 1) // Lu
    pool = int(np.floor(0.8 * units))
    evals = []
    for k in range(3):
        w, ev, perm = oracle.estimation_weights(m, L, 0.8, fixed, 5, 2, k)
        assert sorted(perm.tolist()) == list(range(units))          # bijection
        keys = [oracle.draw(5, 2, 0 if fixed else k, oracle.TAG_SPLIT, u) for u in range(units)]
        assert perm.tolist() == sorted(range(units), key=lambda u: (keys[u], u))
        ev_units = set(perm[pool:].tolist())
        want_ev = np.zeros(m, dtype=np.uint8)
        for u in ev_units:
            want_ev[u * Lu:min(u * Lu + Lu, m)] = 1
        np.testing.assert_array_equal(ev, want_ev)
        assert np.all(w[ev == 1] == 0)                                  # T^k and E^k disjoint
        # T^k: pool draws with replacement from the pool
        d = _numpy_draws(5, 2, k, oracle.TAG_RESAMPLE, pool)
        want = np.zeros(m, dtype=np.int64)
        for r in d:
            u = int(perm[(r * pool) >> 64])
            want[u * Lu:min(u * Lu + Lu, m)] += 1
        np.testing.assert_array_equal(w, want)
        evals.append(ev)
    if fixed:
        assert all(np.array_equal(evals[0], e) for e in evals)
    else:
        assert not np.array_equal(evals[0], evals[1])


# ----------------------------------------------------------------------------
# Moments, Cholesky, lambda grid
# ----------------------------------------------------------------------------
def test_weighted_moments_equal_replicated_rows():
    g = np.random.Generator(np.random.PCG64(1))
    X = g.standard_normal((60, 7))
    Y = g.standard_normal((60, 3))
    w = g.integers(0, 4, size=60).astype(np.uint32)
    G, B, yy = oracle.weighted_moments(X, Y, w, want_yy=True)
    Xr = np.repeat(X, w, axis=0)
    Yr = np.repeat(Y, w, axis=0)
    np.testing.assert_allclose(G, Xr.T @ Xr, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(B, Xr.T @ Yr, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(yy, (Yr ** 2).sum(0), rtol=1e-13)


def test_cholesky_against_numpy_and_non_pd():
    g = np.random.Generator(np.random.PCG64(2))
    M = g.standard_normal((9, 9))
    A = M @ M.T + 0.5 * np.eye(9)
    L, st = oracle.cholesky(A)
    assert st == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)
    b = g.standard_normal(9)
    np.testing.assert_allclose(oracle.cholesky_solve(L, b), np.linalg.solve(A, b), rtol=1e-11)
    A2 = A.copy()
    A2[4, 4] = -1.0
    _, st2 = oracle.cholesky(A2)
    assert st2 < 0


def test_lambda_grid_endpoints():
    lam = oracle.lambda_grid(2.5, 16, 1e-3)
    assert lam[0] == 2.5
    np.testing.assert_allclose(lam[-1], 2.5e-3, rtol=1e-14)
    assert np.all(np.diff(lam) < 0)
    np.testing.assert_allclose(np.diff(np.log10(lam)), -3.0 / 15, rtol=1e-12)
    assert oracle.lambda_grid(1.0, 1)[0] == 1.0


# ----------------------------------------------------------------------------
# LASSO-ADMM (Eq. 2, Eq. 5)
# ----------------------------------------------------------------------------
def _admm_problem(X, y, w=None, rho=1.0):
    G, B = oracle.weighted_moments(X, y, w)
    nk = float(len(y) if w is None else np.sum(w))
    A = G / nk + rho * np.eye(G.shape[0])
    L, st = oracle.cholesky(A)
    assert st == 0
    return G, B[:, 0] / nk, nk, L


def _kkt_bound(G, nk, res, rho, p, tol=1e-6):
    """Bound on the KKT residual of an ADMM exit: s + ||G/nk|| r <= eps_dual + ||G/nk|| eps_pri."""
    x, z, u = res["x"], res["z"], res["u"]
    eps_pri = np.sqrt(p) * tol + tol * max(np.linalg.norm(x), np.linalg.norm(z))
    eps_dual = np.sqrt(p) * tol + tol * rho * np.linalg.norm(u)
    return eps_dual + np.linalg.norm(G / nk, 2) * eps_pri


def test_admm_orthonormal_closed_form():
    g = np.random.Generator(np.random.PCG64(3))
    n, p = 120, 12
    Q, _ = np.linalg.qr(g.standard_normal((n, p)))
    X = np.sqrt(n) * Q                                   # X^T X / n = I
    beta = np.zeros(p)
    beta[[1, 4, 7]] = [2.0, -1.5, 0.7]
    y = X @ beta + 0.3 * g.standard_normal(n)
    G, bn, nk, L = _admm_problem(X, y)
    for lam in [0.01, 0.1, 0.5, 1.0]:
        res = oracle.admm_column(L, bn, lam, max_iter=5000)
        assert res["converged"]
        c = X.T @ y / n
        exact = np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)          # S_lambda(X^T y / n)
        assert np.max(np.abs(res["z"] - exact)) <= 10 * _kkt_bound(G, nk, res, 1.0, p)
        assert set(np.flatnonzero(res["z"])) == set(np.flatnonzero(exact))


def test_admm_zero_above_lambda_max():
    d = synth.workload_data(1)
    lmax = oracle.lambda_max(d.X, d.y)
    assert np.isclose(lmax, np.max(np.abs(d.X.T @ d.y)) / len(d.y), rtol=1e-14)
    G, bn, nk, L = _admm_problem(d.X, d.y)
    res = oracle.admm_column(L, bn, lmax * 1.001, max_iter=5000)
    assert res["converged"]
    assert np.all(res["z"] == 0.0)                     # exactly zero, not just small
    res2 = oracle.admm_column(L, bn, lmax * 0.98, max_iter=5000)
    assert np.count_nonzero(res2["z"]) == 1
    assert np.argmax(np.abs(res2["z"])) == np.argmax(np.abs(bn))


def test_admm_kkt_every_lambda_with_weights():
    d = synth.workload_data(1)
    n, p = d.X.shape
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 16)
    w = oracle.selection_weights(n, 0, 0, 0, 3)
    out = oracle.lasso_admm_batch(d.X, d.y, w[None, :], lam, warm_start=1)
    G, B = oracle.weighted_moments(d.X, d.y, w)
    nk = float(w.sum())
    L, _ = oracle.cholesky(G / nk + np.eye(p))
    z = np.zeros(p)
    u = np.zeros(p)
    for j in range(16):
        beta = out["beta"][0, j, 0]
        res = oracle.admm_column(L, B[:, 0] / nk, lam[j], z0=z, u0=u)
        np.testing.assert_array_equal(res["z"], beta)          # batch == column, same path
        z, u = res["z"], res["u"]
        grad = (B[:, 0] - G @ beta) / nk                       # X^T W (y - X beta) / nk
        tau = _kkt_bound(G, nk, res, 1.0, p) * 1.01
        on = beta != 0
        assert np.all(np.abs(grad[on] - lam[j] * np.sign(beta[on])) <= tau)
        assert np.all(np.abs(grad[~on]) <= lam[j] + tau)


def _brute_force_lasso(X, y, lam, w=None):
    """Exact minimiser of (1/2nk)||y - X b||_W^2 + lam ||b||_1 by enumerating sign patterns."""
    G, B = oracle.weighted_moments(X, y, w)
    b = B[:, 0]
    nk = float(len(y) if w is None else np.sum(w))
    p = X.shape[1]
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
            assert best is None or np.allclose(best, beta, atol=1e-9)
            best = beta
    assert best is not None
    return best


@pytest.mark.parametrize("p,seed", [(5, 0), (7, 1), (8, 2)])
def test_admm_brute_force_small_p(p, seed):
    g = np.random.Generator(np.random.PCG64(100 + seed))
    n = 40
    X = g.standard_normal((n, p))
    beta = np.zeros(p)
    beta[: p // 2] = g.uniform(1, 2, p // 2) * g.choice([-1, 1], p // 2)
    y = X @ beta + 0.5 * g.standard_normal(n)
    w = oracle.selection_weights(n, 0, 0, 0, seed)
    lmax = oracle.lambda_max(X, y)
    lam = oracle.lambda_grid(lmax, 6)
    out = oracle.lasso_admm_batch(X, y, w[None, :], lam, warm_start=1, max_iter=20000)
    G, B = oracle.weighted_moments(X, y, w)
    nk = float(w.sum())
    for j in range(1, 6):
        exact = _brute_force_lasso(X, y, lam[j], w)
        got = out["beta"][0, j, 0]
        assert np.max(np.abs(got - exact)) <= 1e-4 * max(1.0, np.max(np.abs(exact)))
        # identical support except features sitting within 1e-6 of the threshold
        grad = (B[:, 0] - G @ exact) / nk
        ambiguous = (np.abs(np.abs(grad) - lam[j]) <= 1e-6) & (exact == 0)
        ambiguous |= (np.abs(exact) <= 1e-6) & (exact != 0)
        assert np.array_equal((got != 0) | ambiguous, (exact != 0) | ambiguous)


def test_admm_against_sklearn():
    sk = pytest.importorskip("sklearn.linear_model")
    d = synth.workload_data(1)
    n, p = d.X.shape
    w = oracle.selection_weights(n, 0, 0, 0, 1)
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 16)
    out = oracle.lasso_admm_batch(d.X, d.y, w[None, :], lam)
    Xr = np.repeat(d.X, w, axis=0)
    yr = np.repeat(d.y, w)
    for j in [2, 6, 10, 15]:
        m = sk.Lasso(alpha=lam[j], fit_intercept=False, tol=1e-12, max_iter=100000)
        m.fit(Xr, yr)
        np.testing.assert_allclose(out["beta"][0, j, 0], m.coef_, atol=2e-5)


def test_admm_cold_and_path_reach_same_minimiser():
    d = synth.workload_data(1)
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 8)
    a = oracle.lasso_admm_batch(d.X, d.y, None, lam, warm_start=0)
    b = oracle.lasso_admm_batch(d.X, d.y, None, lam, warm_start=1)
    np.testing.assert_allclose(a["beta"], b["beta"], atol=5e-5)
    assert b["iters"].sum() < a["iters"].sum()            # warm start saves iterations


def test_max_iter_flags_non_convergence():
    d = synth.workload_data(1)
    lam = oracle.lambda_grid(oracle.lambda_max(d.X, d.y), 4)
    out = oracle.lasso_admm_batch(d.X, d.y, None, lam, max_iter=1)
    assert out["status"] == oracle.OK_WITH_WARNINGS
    assert not out["conv"].all()
    assert np.all(out["iters"] == 1)


def test_vectorised_var_equals_per_equation_lasso():
    """Eq. 9: the LASSO on (I kron X) vec B splits into p LASSOs sharing X."""
    vp = synth.var_problem(3, 80, 0.4, 0.8, seed=5, burn_in=50)
    S = vp.series
    X, Y = S[:-1], S[1:]
    m, p = X.shape
    K = np.kron(np.eye(p), X)                        # (p m) x (p p), column-stacked vec
    vecY = Y.T.reshape(-1)                           # vec stacks the columns of Y
    lam = oracle.lambda_grid(oracle.lambda_max(X, Y), 5)
    per_eq = oracle.lasso_admm_batch(X, Y, None, lam, warm_start=1, max_iter=20000,
                                     abs_tol=1e-9, rel_tol=1e-9)
    # (1/(2pm))||vecY - K b||^2 + (lam/p)||b||_1 = (1/p) sum_e [per-equation objective]
    vec = oracle.lasso_admm_batch(K, vecY, None, lam / p, warm_start=1, max_iter=20000,
                                  abs_tol=1e-9, rel_tol=1e-9)
    for j in range(5):
        B_vec = vec["beta"][0, j, 0].reshape(p, p)    # column e of B = beta_e
        np.testing.assert_allclose(B_vec, per_eq["beta"][0, j], atol=1e-6)


def test_kronecker_sparsity_printed_value():
    with open(os.path.join(GOLDEN, "kronecker_sparsity.txt")) as f:
        p, pct = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")][0]
    p = int(p)
    X = np.ones((4, p))
    K = np.kron(np.eye(p), X)
    sparsity = 100.0 * (1.0 - np.count_nonzero(K) / K.size)
    assert sparsity == pytest.approx(100.0 * (1.0 - 1.0 / p), rel=1e-14)
    # the paper prints the value cut (not rounded) to two decimals: 98.947 -> 98.94
    assert int(sparsity * 100) / 100 == float(pct)


# ----------------------------------------------------------------------------
# OLS on a support
# ----------------------------------------------------------------------------
def _bits(idx, p):
    W = (p + 63) // 64
    b = np.zeros(W, dtype=np.uint64)
    for i in idx:
        b[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return b


def test_ols_support_against_lstsq():
    g = np.random.Generator(np.random.PCG64(4))
    X = g.standard_normal((50, 70))
    y = g.standard_normal(50)
    w = oracle.selection_weights(50, 0, 1, 0, 0)
    G, B = oracle.weighted_moments(X, y, w)
    S = [0, 3, 17, 63, 64, 69]
    beta, fb = oracle.ols_support(G, B[:, 0], _bits(S, 70))
    assert not fb
    Xr = np.repeat(X[:, S], w, axis=0)
    yr = np.repeat(y, w)
    ref = np.linalg.lstsq(Xr, yr, rcond=None)[0]
    np.testing.assert_allclose(beta[S], ref, rtol=1e-10, atol=1e-12)
    assert np.all(np.delete(beta, S) == 0)
    # residual orthogonal to the support columns
    res = yr - Xr @ beta[S]
    assert np.max(np.abs(Xr.T @ res)) < 1e-9


def test_ols_rank_deficient_min_norm():
    g = np.random.Generator(np.random.PCG64(5))
    X = g.standard_normal((30, 6))
    X[:, 5] = X[:, 2]                          # duplicated column -> singular G[S,S]
    y = g.standard_normal(30)
    G, B = oracle.weighted_moments(X, y)
    S = [1, 2, 5]
    beta, fb = oracle.ols_support(G, B[:, 0], _bits(S, 6))
    assert fb
    ref = np.linalg.lstsq(X[:, S], y, rcond=None)[0]   # minimum-norm solution
    np.testing.assert_allclose(beta[S], ref, rtol=1e-8, atol=1e-10)


def test_ols_empty_support():
    G = np.eye(4)
    beta, fb = oracle.ols_support(G, np.ones(4), np.zeros(1, dtype=np.uint64))
    assert not fb and np.all(beta == 0)


# ----------------------------------------------------------------------------
# Whole fit: intersection (Eq. 3), argmin, union (Eq. 4) and recovery
# ----------------------------------------------------------------------------
def _supports(beta):
    return set(np.flatnonzero(beta).tolist())


def test_fit_set_logic_and_bagging_small():
    d = synth.lasso_problem(80, 9, 3, seed=77, sigma=0.5)
    B1, B2, q = 5, 4, 6
    for bagging in (0, 1):
        out = oracle.uoi_lasso_fit(d.X, d.y, B1, B2, q, bagging=bagging)
        assert out["status"] in (0, 1)
        # Eq. 3: family = intersection of the bootstrap supports (Python sets)
        for j in range(q):
            inter = set(range(9))
            for k in range(B1):
                inter &= _supports(out["sel_beta"][k, j, 0])
            fam = {i for i in range(9)
                   if (int(out["family"][j, 0, i // 64]) >> (i % 64)) & 1}
            assert fam == inter
        # estimation: OLS on S_j, held-out loss, argmin with ties -> smallest j
        n = d.X.shape[0]
        chosen = []
        for k in range(B2):
            wt, ev, _ = oracle.estimation_weights(n, 0, 0.8, 0, 0, 0, k)
            G, B = oracle.weighted_moments(d.X, d.y, wt)
            losses = []
            for j in range(q):
                bj = out["est_beta"][k, j, 0]
                S = sorted(_supports(bj))
                fam = {i for i in range(9)
                       if (int(out["family"][j, 0, i // 64]) >> (i % 64)) & 1}
                assert set(S) <= fam
                if S:
                    Xr = np.repeat(d.X[:, S], wt, axis=0)
                    yr = np.repeat(d.y, wt)
                    np.testing.assert_allclose(bj[S], np.linalg.lstsq(Xr, yr, rcond=None)[0],
                                               rtol=1e-9, atol=1e-11)
                res = d.y[ev == 1] - d.X[ev == 1] @ bj
                losses.append(float(res @ res))
            np.testing.assert_allclose(out["est_loss"][k, :, 0], losses, rtol=1e-12)
            jstar = int(np.argmin(losses))
            assert out["est_jstar"][k] == jstar
            chosen.append(out["est_beta"][k, jstar, 0])
        agg = np.median(chosen, axis=0) if bagging == 0 else np.mean(chosen, axis=0)
        np.testing.assert_allclose(out["beta"][0], agg, rtol=1e-14, atol=1e-15)


def test_fit_noiseless_recovery():
    d = synth.lasso_problem(150, 20, 4, seed=8, sigma=0.0)
    out = oracle.uoi_lasso_fit(d.X, d.y, 8, 6, 12)
    np.testing.assert_allclose(out["beta"][0], d.beta, atol=1e-9)


def test_var_fit_noiseless_permutation_recovery():
    p, T = 6, 60
    g = np.random.Generator(np.random.PCG64(12))
    perm = np.roll(np.arange(p), 1)
    A = np.zeros((p, p))
    A[np.arange(p), perm] = g.choice([-1.0, 1.0], p)
    S = np.zeros((T, p))
    S[0] = g.standard_normal(p)
    for t in range(1, T):
        S[t] = A @ S[t - 1]
    out = oracle.uoi_var_fit(S, 6, 6, 8, block_len=5)
    np.testing.assert_allclose(out["beta"], A, atol=1e-8)


def test_var_fit_is_lagged_lasso_with_joint_argmin():
    vp = synth.var_problem(5, 120, 0.3, 0.8, seed=21, burn_in=50)
    out = oracle.uoi_var_fit(vp.series, 4, 3, 5, block_len=10)
    # per-equation losses sum to the joint loss that picks j*
    for k in range(3):
        assert out["est_jstar"][k] == int(np.argmin(out["est_loss"][k].sum(axis=1)))
    # rows pair X_{t+1} with X_t
    m = vp.series.shape[0] - 1
    X, Y = vp.series[:-1], vp.series[1:]
    lmax = max(np.max(np.abs(X.T @ Y[:, e])) / m for e in range(5))
    np.testing.assert_allclose(out["lambdas"][0], lmax, rtol=1e-13)


def test_fit_argument_errors():
    d = synth.workload_data(1)
    assert oracle.uoi_lasso_fit(d.X, d.y, 0, 2, 3)["status"] == oracle.ERR_INVALID_ARG
    assert oracle.uoi_lasso_fit(d.X, d.y, 2, 2, 3, train_frac=1.0)["status"] == oracle.ERR_INVALID_ARG
    assert oracle.uoi_lasso_fit(d.X, d.y, 2, 2, 3, rho=0.0)["status"] == oracle.ERR_INVALID_ARG
    Xn = d.X.copy()
    Xn[3, 4] = np.nan
    assert oracle.uoi_lasso_fit(Xn, d.y, 2, 2, 3)["status"] == oracle.ERR_NONFINITE
