"""Full-size workloads through the C ABI, checked on sampled outputs (GPU).

At the sizes bench.py times, the oracle cannot redo a whole fit, so it
recomputes sampled pieces one by one from the GPU's own (separately verified)
bootstrap indices:
  * bootstrap indices and eval masks of sampled bootstraps: bit-exact;
  * selection LASSO columns of sampled (bootstrap, equation) paths: the plain
    form against the oracle's ADMM on the oracle's moments (iterations, supports,
    1e-6); the mixed form against the exact minimiser the oracle polishes from its
    ADMM iterate (stopping-rule KKT residual, distance, supports outside the
    band that residual leaves open: mixed_check);
  * family = intersection of the GPU's own per-bootstrap supports (Eq. 3);
  * OLS estimates and held-out losses of sampled (k, j, e) vs the oracle;
  * j* = argmin of the losses summed over equations, beta* = median of the
    chosen estimates (properties that hold at any size).
The UoI_LASSO 50000 x 2000 Gram of a sampled bootstrap is formed with numpy's
matmul (a library primitive) and factored / iterated by the oracle.
"""
import numpy as np
import pytest

import mixed_check
import oracle
from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def bits_to_bool(words, p):
    w = np.asarray(words).astype(np.uint64)
    out = np.zeros(w.shape[:-1] + (p,), dtype=bool)
    for i in range(p):
        out[..., i] = (w[..., i // 64] >> np.uint64(i % 64)) & np.uint64(1)
    return out


def _gpu_fit(X, Y, precision, **kw):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    out = native.uoi_fit_traced(Xd, Yd, precision=precision, **kw)
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def _check_properties(out, p, r):
    B1 = out["sel_beta"].shape[0]
    fam = bits_to_bool(out["family"].astype(np.uint64), p)            # q x r x p
    inter = np.all(out["sel_beta"] != 0, axis=0)                       # q x r x p
    np.testing.assert_array_equal(fam, inter)                          # Eq. 3
    loss = out["est_loss"]                                             # B2 x q x r
    np.testing.assert_array_equal(out["est_jstar"], np.argmin(loss.sum(axis=2), axis=1))
    np.testing.assert_allclose(out["beta"], np.median(out["est_beta"], axis=0), rtol=0, atol=1e-14)
    return fam


@pytest.mark.parametrize("precision", [native.PREC_FP64, native.PREC_MIXED])
def test_var_p192_fullsize_sampled(precision):
    w = synth.WORKLOADS[3]
    vp = synth.workload_data(3)
    S = vp.series
    X, Y = S[:-1], S[1:]
    m, p = X.shape
    kw = dict(B1=w.B1, B2=w.B2, q=w.q, block_len=w.block_len)
    out = _gpu_fit(X, Y, precision, **kw)
    fam = _check_properties(out, p, p)
    # indices of sampled bootstraps
    for k in (0, 17, w.B1 - 1):
        np.testing.assert_array_equal(out["sel_weights"][k],
                                      oracle.selection_weights(m, w.block_len, 0, 0, k))
    for k in (0, w.B2 - 1):
        wt, ev, _ = oracle.estimation_weights(m, w.block_len, 0.8, 0, 0, 0, k)
        np.testing.assert_array_equal(out["est_weights"][k], wt)
        np.testing.assert_array_equal(out["est_eval"][k], ev)
    lam = oracle.lambda_grid(oracle.lambda_max(X, Y), w.q)
    assert rel_l2(out["lambdas"], lam) <= 1e-13
    # selection columns of sampled (bootstrap, equation) paths
    eqs = np.array([0, 101], dtype=np.int64)
    ks = [0, 23]
    wsel = np.stack([out["sel_weights"][k] for k in ks]).astype(np.uint32)
    ref = oracle.lasso_admm_batch(X, Y, wsel, out["lambdas"], warm_start=1, eq_list=eqs)
    if precision == native.PREC_FP64:
        mism = 0
        worst = 0.0
        for a, k in enumerate(ks):
            for j in range(w.q):
                for b, e in enumerate(eqs):
                    g = out["sel_beta"][k, j, e]
                    rz = ref["beta"][a, j, b]
                    worst = max(worst, rel_l2(g, rz))
                    amb = (np.abs(np.abs(ref["v"][a, j, b]) - out["lambdas"][j]) <= 1e-6)
                    amb |= (np.abs(rz) <= 1e-6) & (rz != 0)
                    mism += int(((g != 0) != (rz != 0))[~amb].sum())
        assert worst <= 1e-6, worst
        assert mism == 0
        np.testing.assert_array_equal(out["sel_iters"][ks][:, :, eqs], ref["iters"])
    else:
        rep = mixed_check.check_batch(X, Y, wsel, out["lambdas"], out["sel_beta"], ref["beta"],
                                      mixed_check.ETA_MIXED, ks=ks, eqs=eqs)
        print(rep)
    # estimation: OLS and held-out loss of sampled (k, j, e)
    for k in (0, w.B2 - 1):
        wt = out["est_weights"][k]
        ev = out["est_eval"][k].astype(bool)
        G, B = oracle.weighted_moments(X, Y, wt)
        for j in (0, w.q // 2, w.q - 1):
            for e in eqs:
                bits = out["family"][j, e].astype(np.uint64)
                beta, fb = oracle.ols_support(G, B[:, e], bits)
                res = Y[ev, e] - X[ev] @ beta
                want = float(res @ res)
                ltol = 1e-9 if precision == native.PREC_FP64 else 2e-5
                assert abs(out["est_loss"][k, j, e] - want) <= ltol * max(want, 1e-12)
        jstar = out["est_jstar"][k]
        for e in eqs:
            beta, _ = oracle.ols_support(G, B[:, e], out["family"][jstar, e].astype(np.uint64))
            ctol = 1e-6 if precision == native.PREC_FP64 else 1e-5
            assert rel_l2(out["est_beta"][k, e], beta) <= ctol


def test_lasso_50000x2000_mixed_fullsize_sampled():
    w = synth.WORKLOADS[2]
    d = synth.workload_data(2)
    X, y = d.X, d.y
    n, p = X.shape
    kw = dict(B1=w.B1, B2=w.B2, q=w.q, warm_start=native.WARM_NONE)
    out = _gpu_fit(X, y.reshape(-1, 1), native.PREC_MIXED, **kw)
    _check_properties(out, p, 1)
    k = 5
    wk = oracle.selection_weights(n, 0, 0, 0, k)
    np.testing.assert_array_equal(out["sel_weights"][k], wk)
    lam = out["lambdas"]
    lmax = np.max(np.abs(X.T @ y)) / n                        # numpy matmul as a step
    assert abs(lam[0] - lmax) <= 1e-12 * lmax
    # oracle ADMM on the FP64 Gram of bootstrap k (formed with numpy's matmul)
    Xw = X * wk[:, None].astype(np.float64)
    G = Xw.T @ X
    b = Xw.T @ y
    nk = float(wk.sum())
    L, st = oracle.cholesky(G / nk + np.eye(p))
    assert st == 0
    js = (0, 6, 12, 24, 36, 47)
    z_ref = np.zeros((1, w.q, 1, p))
    for j in js:
        z_ref[0, j, 0] = oracle.admm_column(L, b / nk, lam[j])["z"]     # cold start, as the GPU run
    ev = np.linalg.eigvalsh(G / nk)
    rep = mixed_check.Report()
    for j in js:
        mixed_check.check_column(G, b, nk, lam[j], out["sel_beta"][k, j, 0], z_ref[0, j, 0],
                                 mixed_check.ETA_MIXED, float(ev[0]), float(ev[-1]), rep)
    print(rep)
    # estimation OLS of a sampled bootstrap on the chosen supports, FP64 normal equations
    k2 = 7
    wt = out["est_weights"][k2]
    Xt = X * wt[:, None].astype(np.float64)
    S = np.flatnonzero(bits_to_bool(out["family"][out["est_jstar"][k2], 0].astype(np.uint64), p))
    if len(S):
        Gs = Xt[:, S].T @ X[:, S]
        bs = Xt[:, S].T @ y
        beta = np.zeros(p)
        beta[S] = np.linalg.solve(Gs, bs)
        assert rel_l2(out["est_beta"][k2, 0], beta) <= 1e-5


def test_var2_intercept_p192_fullsize_sampled_mixed():
    # workload 3's series as a VAR(2) with intercept: P = 384 > 192 runs the
    # tensor-core x-update on the eliminated moments of [X~ 1]
    w = synth.WORKLOADS[3]
    S = synth.workload_data(3).series
    N, p = S.shape
    X = np.ascontiguousarray(np.concatenate([S[1:N - 1], S[0:N - 2]], axis=1))
    Y = np.ascontiguousarray(S[2:])
    m, P = X.shape
    kw = dict(B1=w.B1, B2=w.B2, q=w.q, block_len=w.block_len, intercept=1, warm_start=native.WARM_NONE)
    out = _gpu_fit(X, Y, native.PREC_MIXED, **kw)
    assert out["beta"].shape == (p, P + 1)
    _check_properties(out, P, p)
    # selection columns of sampled (bootstrap, equation) pairs vs the oracle's
    # intercept LASSO on the same bootstrap weights
    rep = mixed_check.Report()
    for k in (0, w.B1 - 1):
        wk = out["sel_weights"][k]
        np.testing.assert_array_equal(wk, oracle.selection_weights(m, w.block_len, 0, 0, k))
        for e in (3, 150):
            ref = oracle.lasso_admm_intercept(X, Y[:, e], wk, out["lambdas"], warm_start=0)
            # the selection problem of a fit with an intercept: the w-centred data
            mixed_check.check_batch(X, Y, [wk], out["lambdas"], out["sel_beta"], ref["beta"][None],
                                    mixed_check.ETA_MIXED, ks=[k], eqs=[e], rep=rep, centre=True)
    print(rep)
    # estimation: OLS with the intercept and held-out losses of sampled (k, j, e)
    Xa = np.concatenate([X, np.ones((m, 1))], axis=1)
    Wa = (P + 1 + 63) // 64
    for k in (0, w.B2 - 1):
        wt = out["est_weights"][k]
        ev = out["est_eval"][k].astype(bool)
        G, B = oracle.weighted_moments(Xa, Y, wt)
        for j in (0, w.q // 2, w.q - 1):
            for e in (3, 150):
                bits = np.zeros(Wa, dtype=np.uint64)
                fam = out["family"][j, e].astype(np.uint64)
                bits[:fam.shape[0]] = fam
                bits[P // 64] |= np.uint64(1) << np.uint64(P % 64)
                beta, _ = oracle.ols_support(G, B[:, e], bits)
                res = Y[ev, e] - Xa[ev] @ beta
                want = float(res @ res)
                assert abs(out["est_loss"][k, j, e] - want) <= 2e-5 * max(want, 1e-12)


def test_var_p1000_fullsize_sampled_mixed():
    # workload 5 (VAR(1), p = 1000, T = 20000, B1 = B2 = 32, q = 40) in the mixed form
    # with path warm start (its fastest schedule): bootstrap indices of sampled
    # bootstraps bit-exact; selection columns of sampled (bootstrap, equation) paths
    # against the exact minimiser; the intersection / argmin / median properties;
    # OLS and held-out losses of sampled (k, j, e) against the oracle
    w = synth.WORKLOADS[5]
    S = synth.workload_data(5).series
    X, Y = np.ascontiguousarray(S[:-1]), np.ascontiguousarray(S[1:])
    m, p = X.shape
    kw = dict(B1=w.B1, B2=w.B2, q=w.q, block_len=w.block_len, warm_start=native.WARM_PATH)
    out = _gpu_fit(X, Y, native.PREC_MIXED, **kw)
    _check_properties(out, p, p)
    ks, eqs = [w.B1 - 1], [7, 512]
    for k in (0, w.B1 - 1):
        np.testing.assert_array_equal(out["sel_weights"][k], oracle.selection_weights(m, w.block_len, 0, 0, k))
    conv = out["sel_conv"][ks][:, :, eqs]
    wsel = np.stack([out["sel_weights"][k] for k in ks]).astype(np.uint32)
    ref = oracle.lasso_admm_batch(X, np.ascontiguousarray(Y[:, eqs]), wsel, out["lambdas"], warm_start=1,
                                  max_iter=5000)
    assert ref["conv"].all()
    # columns the GPU finished within max_iter: held to the exact minimiser
    rep = mixed_check.Report()
    for a, k in enumerate(ks):
        G, Bm, nk = mixed_check.moments(X, Y[:, eqs], out["sel_weights"][k])
        ev = np.linalg.eigvalsh(G / nk)
        for b, e in enumerate(eqs):
            for j in range(w.q):
                if not conv[a, j, b]:
                    continue
                mixed_check.check_column(G, Bm[:, b], nk, out["lambdas"][j], out["sel_beta"][k, j, e],
                                         ref["beta"][a, j, b], mixed_check.ETA_MIXED, float(ev[0]),
                                         float(ev[-1]), rep)
    print(rep, f"; columns stopped at max_iter: {int((~conv.astype(bool)).sum())} of {conv.size}")
    assert rep.columns >= conv.size // 2
    for k in (w.B2 - 1,):
        wt = out["est_weights"][k]
        ev = out["est_eval"][k].astype(bool)
        G, B, _ = mixed_check.moments(X, Y[:, eqs], wt)
        for j in (0, w.q // 2, w.q - 1):
            for b, e in enumerate(eqs):
                beta, _ = oracle.ols_support(G, B[:, b], out["family"][j, e].astype(np.uint64))
                res = Y[ev, e] - X[ev] @ beta
                want = float(res @ res)
                assert abs(out["est_loss"][k, j, e] - want) <= 2e-5 * max(want, 1e-12)
