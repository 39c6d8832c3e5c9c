"""Weighted moments (G1) through the C ABI against the oracle's triple loops (GPU).

FP64 CUDA-core form: within 1e-13 of the largest entry.  Tensor-core form
(split bf16, FP32 tensor-core accumulation per 128 rows, compensated sums):
within 2e-6 of the largest diagonal entry, the budget derived in gram_tc.cu
(<= 5e-7 from 24 truncating accumulation steps, 2^-17 split residue and the
zero-mean off-diagonal lo*lo term averaged over the sample).  Sizes span several 128 x 256 tiles, ragged feature counts
and a sample longer than one accumulation chunk.
"""
import numpy as np
import pytest

import oracle
from paper_1808_06992_gb300 import native

pytestmark = pytest.mark.gpu


def _case(n, p, r, B, seed, wmax=4):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((n, p))
    Y = g.standard_normal((n, r))
    w = np.stack([oracle.selection_weights(n, 0, seed, 0, k) for k in range(B)])
    if wmax is not None:
        w[0] = g.integers(0, wmax, size=n)
    return X, Y, w.astype(np.uint32)


# Row tiles of 128 run in pairs (2m, 2m+1) on one 256-column tile: odd counts of
# row tiles (51, 78, 301, 516, 520 columns of Z) leave the last pair's second tile
# past the end; 251 and 1101 columns give even and odd counts with several column
# tiles per pair.
@pytest.mark.parametrize("n,p,r,B", [(200, 50, 1, 3), (1000, 77, 1, 2), (5000, 300, 1, 2),
                                     (9000, 513, 3, 1), (700, 260, 260, 2), (3000, 250, 1, 2),
                                     (2500, 1100, 1, 1)])
def test_moments_fp64_and_tc_vs_oracle(n, p, r, B):
    X, Y, w = _case(n, p, r, B, seed=n + p)
    G64, B64 = native.weighted_moments(X, Y, w, precision=native.PREC_FP64)
    Gtc, Btc = native.weighted_moments(X, Y, w, precision=native.PREC_MIXED)
    for k in range(B):
        Gr, Br = oracle.weighted_moments(X, Y, w[k])
        scale = np.max(np.abs(np.diag(Gr)))
        assert np.max(np.abs(G64[k] - Gr)) <= 1e-13 * scale
        assert np.max(np.abs(B64[k] - Br)) <= 1e-13 * scale
        assert np.array_equal(Gtc[k], Gtc[k].T)                      # exactly symmetric
        assert np.max(np.abs(Gtc[k] - Gr)) <= 2e-6 * scale
        yscale = max(scale, np.max(np.abs(Br)))
        assert np.max(np.abs(Btc[k] - Br)) <= 2e-6 * yscale


def test_moments_tc_zero_weight_rows_and_single_row():
    X, Y, _ = _case(300, 40, 1, 1, seed=3)
    w = np.zeros((2, 300), dtype=np.uint32)
    w[0, 17] = 3                       # one row, weight 3
    w[1, :] = 1
    Gtc, Btc = native.weighted_moments(X, Y, w, precision=native.PREC_MIXED)
    # a single row: the off-diagonal lo*lo term (<= 2^-16 relative) does not average out
    np.testing.assert_allclose(Gtc[0], 3.0 * np.outer(X[17], X[17]), rtol=4e-5, atol=1e-12)
    Gr, Br = oracle.weighted_moments(X, Y, w[1])
    assert np.max(np.abs(Gtc[1] - Gr)) <= 2e-6 * np.max(np.diag(Gr))


def test_moments_tc_item_without_rows():
    # an item whose weights are all zero has no sample rows: its moments are exactly zero,
    # and the other items of the same launch are unaffected
    X, Y, w = _case(2000, 300, 1, 3, seed=11)
    w[1, :] = 0
    Gtc, Btc = native.weighted_moments(X, Y, w, precision=native.PREC_MIXED)
    assert not Gtc[1].any() and not Btc[1].any()
    for k in (0, 2):
        Gr, Br = oracle.weighted_moments(X, Y, w[k])
        scale = np.max(np.abs(np.diag(Gr)))
        assert np.max(np.abs(Gtc[k] - Gr)) <= 2e-6 * scale
        assert np.max(np.abs(Btc[k] - Br)) <= 2e-6 * max(scale, np.max(np.abs(Br)))
