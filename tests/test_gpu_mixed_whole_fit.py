"""Whole UoI_LASSO fits on the code path of the 50000 x 2000 workload, against the oracle (GPU).

X 6000 x 640 with Toeplitz(0.5) rows, 32 nonzeros, SNR 5, B1 = B2 = 6, q = 12,
cold lambda batch (as bench.py runs).  At p = 640 the mixed form runs every
kernel the 2000-feature workload runs: the two-piece bf16 tensor-core Gram,
the block Schur-complement inverse on tensor-core GEMMs (p >= 512), the
tensor-core x-update (p > 192) and the FP32-factor + FP64-refinement OLS on
the union-restricted tensor-core moments.

  * plain FP64 form: the full trace against the oracle (indices, iterations,
    supports, family and j* bit-exact, coefficients within 1e-6);
  * mixed form: every selection column held to the exact minimiser (the
    oracle's ADMM iterate polished; mixed_check), the family identical to the
    oracle's outside the bits whose intersection touched a band feature
    (counted), and then j* identical and the bagged beta* (Alg. 1's output)
    within 1e-5 relative l2 of the oracle's.
"""
import numpy as np
import pytest

import mixed_check
import oracle
from paper_1808_06992_gb300 import native, synth
from test_gpu_parity import bits_to_bool, compare_fit, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = dict(B1=6, B2=6, q=12, warm_start=0)


def _problem():
    return synth.lasso_problem(6000, 640, 32, seed=61, snr=5.0, mag=(0.5, 3.0), toeplitz_rho=0.5)


def _gpu(d, precision):
    Xd = torch.from_numpy(d.X).cuda()
    yd = torch.from_numpy(d.y.reshape(-1, 1)).cuda()
    out = native.uoi_fit_traced(Xd, yd, precision=precision, **KW)
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


@pytest.fixture(scope="module")
def ref():
    d = _problem()
    return d, oracle.uoi_lasso_fit(d.X, d.y, n_threads=8, **KW)


def test_fp64_form_p640_full_trace(ref):
    d, r = ref
    gpu = _gpu(d, native.PREC_FP64)
    rep = compare_fit(r, gpu, d.X, d.y.reshape(-1, 1), **KW)
    assert rep["family_clean"]


def test_mixed_form_p640_whole_fit_within_1e5(ref):
    d, r = ref
    gpu = _gpu(d, native.PREC_MIXED)
    p = d.X.shape[1]
    B1, q = KW["B1"], KW["q"]
    np.testing.assert_array_equal(gpu["sel_weights"], np.stack(
        [oracle.selection_weights(d.X.shape[0], 0, 0, 0, k) for k in range(B1)]))
    assert rel_l2(gpu["lambdas"], r["lambdas"]) <= 1e-13
    assert gpu["sel_conv"].all()
    # selection: every column against the exact minimiser
    rep = mixed_check.check_batch(d.X, d.y, gpu["sel_weights"], r["lambdas"], gpu["sel_beta"],
                                  r["sel_beta"], mixed_check.ETA_MIXED)
    print(rep)
    # family (Eq. 3): identical outside the bits whose intersection touched a band feature
    touched = np.zeros((q, p), dtype=bool)
    for (k, j, e), band in rep.bands.items():
        touched[j] |= band
    fam_g = bits_to_bool(gpu["family"], p)[:, 0, :]
    fam_r = bits_to_bool(r["family"], p)[:, 0, :]
    assert np.array_equal(fam_g | touched, fam_r | touched)
    differ = int((fam_g != fam_r).sum())
    print(f"family bits touched by the band: {int(touched.sum())}, differing: {differ}")
    if differ == 0:
        np.testing.assert_array_equal(gpu["est_jstar"], r["est_jstar"])
        # held-out losses from the tensor-core moments (elementwise 2e-6 of the largest
        # diagonal) and the FP64-accurate OLS
        np.testing.assert_allclose(gpu["est_loss"], r["est_loss"], rtol=1e-5)
        err = rel_l2(gpu["beta"][0], r["beta"][0])
        print(f"beta* rel l2 vs the oracle: {err:.2e}")
        assert err <= 1e-5
    else:
        pytest.fail(f"{differ} family bits differ (inside the band): no beta* statement")
