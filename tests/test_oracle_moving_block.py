"""Pins of the oracle's moving-block selection bootstrap (Kunsch's overlapping
blocks, the alternative to the non-overlapping blocks of Sec. III-A-2):
its exact block structure, its reduction to the row bootstrap, and the
coverage profile implied by uniform block starts."""
import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import synth


def _starts_from_coverage(w, L):
    """Block-start counts h from coverage w = sum of L-row indicators:
    w_i = h_{i-L+1} + ... + h_i, so h_i = w_i - w_{i-1} + h_{i-L}."""
    m = w.shape[0]
    h = np.zeros(m, dtype=np.int64)
    for i in range(m):
        h[i] = int(w[i]) - (int(w[i - 1]) if i > 0 else 0) + (h[i - L] if i >= L else 0)
    return h


@pytest.mark.parametrize("m,L", [(997, 10), (500, 1), (123, 123), (1000, 37)])
def test_moving_blocks_are_whole_runs_of_L_rows(m, L):
    for k in range(3):
        w = oracle.selection_weights_moving(m, L, 5, 2, k)
        units = -(-m // max(L, 1))
        assert int(w.sum()) == units * max(L, 1)
        h = _starts_from_coverage(w, max(L, 1))
        assert np.all(h >= 0)
        assert np.all(h[m - max(L, 1) + 1:] == 0)          # no block runs past the last row
        assert int(h.sum()) == units


def test_moving_blocks_of_one_row_are_the_row_bootstrap():
    for k in range(3):
        np.testing.assert_array_equal(oracle.selection_weights_moving(400, 1, 9, 1, k),
                                      oracle.selection_weights(400, 1, 9, 1, k))
        np.testing.assert_array_equal(oracle.selection_weights_moving(400, 0, 9, 1, k),
                                      oracle.selection_weights(400, 0, 9, 1, k))


def test_moving_block_coverage_profile():
    # uniform starts on 0..m-L: row i is covered by min(i, m-L) - max(0, i-L+1) + 1 of
    # the m-L+1 start positions, so E[w_i] = units * that / (m - L + 1)
    m, L, B = 300, 20, 4000
    units = -(-m // L)
    mean = np.zeros(m)
    for k in range(B):
        mean += oracle.selection_weights_moving(m, L, 3, 0, k)
    mean /= B
    i = np.arange(m)
    cover = np.minimum(i, m - L) - np.maximum(0, i - L + 1) + 1
    expect = units * cover / (m - L + 1)
    # per-row standard error below ~0.02 at B = 4000
    assert np.max(np.abs(mean - expect)) < 0.08
    assert mean[0] < 0.2 * mean[m // 2]                     # the edges are rarely covered


def test_fit_with_moving_blocks_runs_and_differs_only_in_selection():
    vp = synth.var_problem(6, 300, 0.3, 0.8, seed=17, burn_in=50)
    a = oracle.uoi_var_fit(vp.series, 4, 3, 6, block_len=20)
    b = oracle.uoi_var_fit(vp.series, 4, 3, 6, block_len=20, block_mode=1)
    assert a["status"] >= 0 and b["status"] >= 0
    # estimation samples are the same; the selection bootstraps are not
    np.testing.assert_array_equal(a["eval_count"], b["eval_count"])
    assert not np.array_equal(a["sel_iters"], b["sel_iters"]) or not np.array_equal(a["sel_beta"], b["sel_beta"])
