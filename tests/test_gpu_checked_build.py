"""The checked build: index checks in the kernels, a stand-in for a memory checker (GPU).

The library can be built with UOI_BOUNDS_CHECK=1 (build(checked=True)): the
main stores of the Gram, ADMM, x-update and operand-split kernels check their
index against the extent of the buffer they write; a failed check records
UOI_ERR_BOUNDS in a device status word and skips the access (nothing traps), and
the fit then returns UOI_ERR_BOUNDS.  The tests run the check itself on in-range
and out-of-range indices, and fits through the checked build on the paths of the
precision forms (FP64; mixed with the tensor-core Gram, x-update and Schur
inverse), which must pass every check and equal the release build bit for bit.
"""
import numpy as np
import pytest

from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_index_check_records_and_skips():
    assert native.selftest_index_check(5, 16) == native.OK
    assert native.selftest_index_check(15, 16) == native.OK
    for bad in (16, 1000, -1):
        with pytest.raises(native.UoiError) as ei:
            native.selftest_index_check(bad, 16)
        assert ei.value.status == native.ERR_BOUNDS
        assert "access skipped" in native.last_error()
    assert native.selftest_index_check(0, 1) == native.OK          # the context is still usable


@pytest.mark.parametrize("case", ["fp64", "mixed_p300", "mixed_p640"])
def test_checked_build_passes_and_matches_release(case):
    if case == "fp64":
        d = synth.workload_data(1)
        kw = dict(B1=8, B2=5, q=10, precision=native.PREC_FP64)
    elif case == "mixed_p300":
        d = synth.lasso_problem(1200, 300, 20, seed=31, sigma=0.5, toeplitz_rho=0.5)
        kw = dict(B1=4, B2=3, q=8, precision=native.PREC_MIXED, warm_start=native.WARM_NONE)
    else:
        d = synth.lasso_problem(3000, 640, 30, seed=61, sigma=0.5, toeplitz_rho=0.5)
        kw = dict(B1=3, B2=3, q=6, precision=native.PREC_MIXED, warm_start=native.WARM_NONE)
    rel = native.uoi_fit_traced(d.X, d.y, **kw)
    with native.use_library(native.checked_lib()):
        chk = native.uoi_fit_traced(d.X, d.y, **kw)
    assert chk["status"] == rel["status"]
    for key in ("beta", "sel_beta", "family", "est_loss", "est_jstar"):
        np.testing.assert_array_equal(chk[key], rel[key])
