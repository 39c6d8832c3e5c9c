"""Batched uneven UoI_LASSO problems through uoi_lasso_fit_batch (GPU).

* every problem's result is bitwise the result of uoi_lasso_fit on that problem
  alone with problem_id = base + i (the batch only schedules; the arithmetic is
  the same), in both precision forms, with more problems than worker streams;
* the plain FP64 batch matches the FP64 oracle on its problems (Alg. 1 per
  problem) within the plain form's 1e-6;
* an empty batch and a failing member are reported per problem.
"""
import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu

SIZES = [(300, 20, 4), (1200, 150, 12), (800, 64, 6), (2000, 260, 20), (500, 35, 5), (1500, 100, 8),
         (640, 700, 30)]      # the last has n < p and p >= 512 (tensor-core inverse in the mixed form)


def _problems(sizes):
    return [synth.lasso_problem(n, p, k, seed=4000 + i, sigma=1.0) for i, (n, p, k) in enumerate(sizes)]


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


@pytest.mark.parametrize("prec", [native.PREC_MIXED, native.PREC_FP64])
def test_batch_equals_single_fits(prec):
    probs = _problems(SIZES if prec == native.PREC_MIXED else SIZES[:6])
    kw = dict(B1=6, B2=5, q=8, precision=prec, problem_id=11, warm_start=native.WARM_NONE)
    out = native.uoi_lasso_fit_batch([d.X for d in probs], [d.y for d in probs], streams=3, **kw)
    assert len(out) == len(probs)
    for i, d in enumerate(probs):
        one = native.uoi_lasso_fit(d.X, d.y, **{**kw, "problem_id": 11 + i})
        assert out[i]["status"] in (native.OK, native.OK_WITH_WARNINGS)
        np.testing.assert_array_equal(out[i]["beta"], one["beta"])
        assert out[i]["diag"]["admm_iterations"] == one["diag"]["admm_iterations"]


def test_fp64_batch_matches_oracle():
    probs = _problems(SIZES[:3])
    kw = dict(B1=5, B2=4, q=6, problem_id=3)
    out = native.uoi_lasso_fit_batch([d.X for d in probs], [d.y for d in probs], streams=2,
                                     precision=native.PREC_FP64, **kw)
    for i, d in enumerate(probs):
        ref = oracle.uoi_lasso_fit(d.X, d.y, **{**kw, "problem_id": 3 + i})
        assert rel_l2(out[i]["beta"], ref["beta"][0]) <= 1e-6


def test_empty_and_failing_members():
    assert native.uoi_lasso_fit_batch([], [], B1=2, B2=2, q=2) == []
    good = synth.lasso_problem(200, 10, 3, seed=5, sigma=0.5)
    bad = good.X.copy()
    bad[3, 2] = np.nan
    with pytest.raises(native.UoiError) as ei:
        native.uoi_lasso_fit_batch([good.X, bad], [good.y, good.y], B1=2, B2=2, q=3)
    assert ei.value.status == native.ERR_NONFINITE
