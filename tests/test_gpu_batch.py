"""Batched uneven UoI_LASSO problems through uoi_lasso_fit_batch (GPU).

* every problem's result is bitwise the result of uoi_lasso_fit on that problem
  alone with problem_id = base + i (the batch only schedules; the arithmetic is
  the same), in both precision forms, with more problems than worker streams,
  and in the grouped form (streams = 0: the tensor-core ADMM solves of all
  members iterated together, tiles chosen by timing), whose first call tunes and
  whose second reuses the choice -- both bitwise the single fits, with cold and
  with path warm starts;
* the plain FP64 batch matches the FP64 oracle on its problems (Alg. 1 per
  problem) within the plain form's 1e-6;
* every mixed member (p from 20 to 700, the last with n < p on the tensor-core
  inverse) against the oracle: where the bootstrap problems are strongly convex
  (n > 2p) the selection columns are held to the exact minimiser, the family is
  identical outside the band-touched bits, and beta* is within 1e-5; where
  n <= 2p (a singular bootstrap Gram: the minimiser need not be unique and the
  stopping rule decides no support) every column's KKT residual is held to the
  stopping bound and family differences are reported;
* an empty batch and a failing member are reported per problem.
"""
import numpy as np
import pytest

import mixed_check
import oracle
from paper_1808_06992_gb300 import native, synth
from test_gpu_parity import bits_to_bool

pytestmark = pytest.mark.gpu

SIZES = [(300, 20, 4), (1200, 150, 12), (800, 64, 6), (2000, 260, 20), (500, 35, 5), (1500, 100, 8),
         (640, 700, 30)]      # the last has n < p and p >= 512 (tensor-core inverse in the mixed form)


def _problems(sizes):
    return [synth.lasso_problem(n, p, k, seed=4000 + i, sigma=1.0) for i, (n, p, k) in enumerate(sizes)]


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


@pytest.mark.parametrize("prec,streams", [(native.PREC_MIXED, 3), (native.PREC_FP64, 3), (native.PREC_MIXED, 0),
                                          (native.PREC_FP64, 0)])
def test_batch_equals_single_fits(prec, streams):
    probs = _problems(SIZES if prec == native.PREC_MIXED else SIZES[:6])
    kw = dict(B1=6, B2=5, q=8, precision=prec, problem_id=11, warm_start=native.WARM_NONE)
    runs = [native.uoi_lasso_fit_batch([d.X for d in probs], [d.y for d in probs], streams=streams, **kw)
            for _ in range(2 if streams == 0 else 1)]
    for out in runs:
        assert len(out) == len(probs)
        for i, d in enumerate(probs):
            one = native.uoi_lasso_fit(d.X, d.y, **{**kw, "problem_id": 11 + i})
            assert out[i]["status"] in (native.OK, native.OK_WITH_WARNINGS)
            np.testing.assert_array_equal(out[i]["beta"], one["beta"])
            assert out[i]["diag"]["admm_iterations"] == one["diag"]["admm_iterations"]


def test_grouped_batch_path_warm_start():
    # path warm start: chains advance through the lambdas inside the grouped check
    probs = _problems(SIZES[1:4] + SIZES[6:])
    kw = dict(B1=4, B2=4, q=6, precision=native.PREC_MIXED, problem_id=5, warm_start=native.WARM_PATH)
    out = native.uoi_lasso_fit_batch([d.X for d in probs], [d.y for d in probs], streams=0, **kw)
    for i, d in enumerate(probs):
        one = native.uoi_lasso_fit(d.X, d.y, **{**kw, "problem_id": 5 + i})
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


@pytest.mark.parametrize("streams", [3, 0])
def test_mixed_batch_members_match_oracle(streams):
    probs = _problems(SIZES)
    kw = dict(B1=6, B2=5, q=8, warm_start=native.WARM_NONE)
    out = native.uoi_lasso_fit_batch([d.X for d in probs], [d.y for d in probs], streams=streams,
                                     precision=native.PREC_MIXED, problem_id=11, **kw)
    for i, d in enumerate(probs):
        n, p = d.X.shape
        pid = 11 + i
        ref = oracle.uoi_lasso_fit(d.X, d.y, problem_id=pid, n_threads=8, **kw)
        tr = native.uoi_fit_traced(d.X, d.y, precision=native.PREC_MIXED, problem_id=pid, **kw)
        np.testing.assert_array_equal(out[i]["beta"], tr["beta"][0])     # the member is the single fit
        np.testing.assert_array_equal(tr["sel_weights"], np.stack(
            [oracle.selection_weights(n, 0, 0, pid, k) for k in range(kw["B1"])]))
        fam_g = bits_to_bool(tr["family"], p)[:, 0, :]
        fam_r = bits_to_bool(ref["family"], p)[:, 0, :]
        touched = np.zeros_like(fam_r)
        if n <= 2 * p:
            rep = mixed_check.check_residuals(d.X, d.y, tr["sel_weights"], ref["lambdas"], tr["sel_beta"],
                                              mixed_check.ETA_MIXED)
            print(f"problem {i} ({n} x {p}): {rep}; family bits differing from the oracle: "
                  f"{int((fam_g != fam_r).sum())} of {int(fam_r.sum())}")
            continue
        rep = mixed_check.check_batch(d.X, d.y, tr["sel_weights"], ref["lambdas"], tr["sel_beta"],
                                      ref["sel_beta"], mixed_check.ETA_MIXED)
        for (k, j, e), band in rep.bands.items():
            touched[j] |= band
        print(f"problem {i} ({n} x {p}): {rep}")
        assert np.array_equal(fam_g | touched, fam_r | touched), f"problem {i}: family differs"
        if np.array_equal(fam_g, fam_r):
            np.testing.assert_array_equal(tr["est_jstar"], ref["est_jstar"])
            err = rel_l2(out[i]["beta"], ref["beta"][0])
            print(f"problem {i} ({n} x {p}): beta* rel l2 {err:.2e}")
            assert err <= 1e-5


def test_empty_and_failing_members():
    assert native.uoi_lasso_fit_batch([], [], B1=2, B2=2, q=2) == []
    good = synth.lasso_problem(200, 10, 3, seed=5, sigma=0.5)
    bad = good.X.copy()
    bad[3, 2] = np.nan
    with pytest.raises(native.UoiError) as ei:
        native.uoi_lasso_fit_batch([good.X, bad], [good.y, good.y], B1=2, B2=2, q=3)
    assert ei.value.status == native.ERR_NONFINITE
    # grouped: members that reach the tensor-core solve still finish beside a failing one
    big = synth.lasso_problem(900, 260, 10, seed=6, sigma=0.5)
    bad2 = big.X.copy()
    bad2[0, 0] = np.inf
    with pytest.raises(native.UoiError) as ei:
        native.uoi_lasso_fit_batch([big.X, bad2, big.X], [big.y, big.y, big.y], streams=0, B1=3, B2=2, q=4,
                                   precision=native.PREC_MIXED, problem_id=9)
    assert ei.value.status == native.ERR_NONFINITE
