"""Fault paths through the C ABI, made without faulting the GPU (GPU).

Every mbarrier wait of the tensor-core kernels is bounded; a wait that runs out
makes the kernel record UOI_ERR_TIMEOUT and return, so the call reports the
error and the context stays usable.  uoi_selftest_wait runs that bounded wait
on an mbarrier that nothing arrives on, with a short limit.  No wait here is
unbounded, nothing traps, and no access leaves its buffer.
"""
import numpy as np
import pytest

from paper_1808_06992_gb300 import native, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_runs_out_reports_timeout_and_leaves_the_context_usable():
    limit_ms = 50.0
    with pytest.raises(native.UoiError) as ei:
        native.selftest_wait(int(limit_ms * 1e6), arrive=False)
    assert ei.value.status == native.ERR_TIMEOUT
    assert "ran out" in native.last_error()
    # the wait gave up once the limit had passed, not much later
    assert limit_ms <= ei.value.waited_ms < limit_ms + 500.0
    # the context is still usable: the arriving variant, then a whole fit
    assert native.selftest_wait(int(limit_ms * 1e6), arrive=True) < limit_ms
    d = synth.workload_data(1)
    out = native.uoi_fit_traced(d.X, d.y, B1=4, B2=3, q=6)
    assert out["status"] in (native.OK, native.OK_WITH_WARNINGS)
    assert np.isfinite(out["beta"]).all()


def test_bounded_wait_limit_is_validated():
    for bad in (0, 20 * 10 ** 9):
        with pytest.raises(native.UoiError) as ei:
            native.selftest_wait(bad)
        assert ei.value.status == native.ERR_INVALID_ARG
