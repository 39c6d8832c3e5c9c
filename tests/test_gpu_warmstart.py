"""Learned warm start (GPU): kernels vs the FP64 reference, training, gain, judge.

* forward and loss gradient of the CUDA network (hidden layers on tcgen05 with
  BF16 weights and activations) vs oracle/mlp.py (FP64) on BF16-representable
  weights, with the reference rounding its hidden activations and
  back-propagated gradients to BF16 where the GPU stores them: both then agree
  to the FP32 accumulation and the rare BF16 rounding that FP32 and FP64 values
  decide differently (bound 5e-4 relative);
* training on rows from the method's own path-warm ADMM solutions (problems
  with seeds disjoint from the test problem) lowers the loss;
* on the test problem the learned start needs fewer ADMM iterations than the
  cold start, converges to the same minimiser (KKT gap no worse than the
  path-warm judge's), and a missing weights file falls back to path warm start.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu


def bf16_round(a):
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def _batch(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    X = (g.standard_normal((n, 8)) * 1.5).astype(np.float32)
    T = np.column_stack([g.standard_normal(n), g.uniform(-1, 1, n), g.integers(0, 2, n)]).astype(np.float32)
    return X, T


def test_forward_and_gradient_match_fp64_reference():
    m = native.WarmStartModel(seed=3)
    params = bf16_round(m.get_params())
    m.set_params(params)
    X, T = _batch(300, 11)
    P = mlp.unflatten(params.astype(np.float64))
    ref, _ = mlp.forward(P, X.astype(np.float64), round_act=mlp.bf16_round)
    out = m.forward(X)
    assert rel_l2(out.astype(np.float64), ref) <= 5e-4
    L, g = m.loss_grad(X, T)
    Lr, gr = mlp.loss_and_grad(P, X.astype(np.float64), T.astype(np.float64), round_act=mlp.bf16_round)
    assert abs(L - Lr) <= 5e-5 * abs(Lr)
    flat = mlp.flatten(gr)
    o = 0
    for sh in mlp.shapes():
        n = int(np.prod(sh))
        err = rel_l2(g[o:o + n].astype(np.float64), flat[o:o + n])
        print(sh, f"{err:.2e}")
        assert err <= 5e-4, sh
        o += n


def _training_rows(count, B=8, q=16):
    feats, targs = [], []
    for s in range(count):
        seed = 50000 + s                                   # disjoint from workload 1's seed 1001
        d = synth.lasso_problem(200, 50, 10, seed=seed, sigma=0.5)
        g = np.random.Generator(np.random.PCG64(seed))
        w = np.stack([g.multinomial(200, np.full(200, 1 / 200)) for _ in range(B)]).astype(np.uint32)
        lmax = np.max(np.abs(d.X.T @ d.y)) / 200
        lam = lmax * 10.0 ** (-3.0 * np.arange(q) / (q - 1))
        F, T = native.ws_dataset(d.X, d.y, w, lam)
        feats.append(F)
        targs.append(T)
    return np.concatenate(feats), np.concatenate(targs)


def _kkt_gap(X, y, w, lam, beta):
    """max over features of the LASSO optimality violation for each column."""
    G, B = oracle.weighted_moments(X, y, w)
    nk = float(w.sum())
    gap = 0.0
    for j, bj in enumerate(beta):
        grad = (B[:, 0] - G @ bj) / nk
        on = bj != 0
        gap = max(gap, float(np.max(np.abs(grad[on] - lam[j] * np.sign(bj[on])), initial=0.0)),
                  float(np.max(np.abs(grad[~on]) - lam[j], initial=0.0)))
    return gap


def test_learned_warm_start_trains_gains_and_is_judged(tmp_path):
    F, T = _training_rows(24)
    m = native.WarmStartModel(seed=1)
    L0, _ = m.loss_grad(F[:8192], T[:8192])
    L1 = m.train(F, T, epochs=6, batch=2048, lr=1e-3, seed=5)
    assert L1 < 0.5 * L0, (L0, L1)
    path = str(tmp_path / "ws.bin")
    m.save(path)
    m2 = native.WarmStartModel(path=path)                  # save/load round trip
    np.testing.assert_array_equal(m2.get_params(), m.get_params())

    d = synth.workload_data(1)
    kw = dict(B1=20, B2=10, q=16)
    cold = native.uoi_fit_traced(d.X, d.y, warm_start=native.WARM_NONE, **kw)
    pw = native.uoi_fit_traced(d.X, d.y, warm_start=native.WARM_PATH, **kw)
    lw = native.uoi_fit_traced(d.X, d.y, warm_start=native.WARM_LEARNED, mlp_weights_path=path, **kw)
    assert lw["diag"]["warm_start_used"] == native.WARM_LEARNED
    it_cold, it_path, it_learned = (int(o["sel_iters"].sum()) for o in (cold, pw, lw))
    print(f"ADMM iterations: cold {it_cold}, path {it_path}, learned {it_learned}")
    assert it_learned < 0.95 * it_cold               # measured: about 10 % fewer than cold
    # judge: the learned start reaches the same minimiser as path warm start
    lam = pw["lambdas"]
    worst_l, worst_p = 0.0, 0.0
    for k in range(0, 20, 4):
        w = pw["sel_weights"][k]
        worst_l = max(worst_l, _kkt_gap(d.X, d.y, w, lam, lw["sel_beta"][k, :, 0]))
        worst_p = max(worst_p, _kkt_gap(d.X, d.y, w, lam, pw["sel_beta"][k, :, 0]))
    assert worst_l <= 2.0 * worst_p + 1e-5, (worst_l, worst_p)
    np.testing.assert_array_equal(lw["family"], pw["family"])
    assert rel_l2(lw["beta"], pw["beta"]) <= 1e-5


def test_missing_weights_fall_back_to_path():
    d = synth.workload_data(1)
    kw = dict(B1=4, B2=3, q=6)
    pw = native.uoi_fit_traced(d.X, d.y, warm_start=native.WARM_PATH, **kw)
    fb = native.uoi_fit_traced(d.X, d.y, warm_start=native.WARM_LEARNED,
                               mlp_weights_path="/nonexistent/ws.bin", **kw)
    assert fb["diag"]["warm_start_used"] == native.WARM_PATH
    np.testing.assert_array_equal(fb["beta"], pw["beta"])
    np.testing.assert_array_equal(fb["sel_iters"], pw["sel_iters"])
