"""Pins of the FP64 reference MLP (CPU only): finite differences, GELU, BCE."""
import math

import numpy as np

from oracle import mlp


def _params(f_in, hidden, f_out, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return [g.standard_normal(sh) * (0.5 / math.sqrt(sh[-1])) if len(sh) == 2 else
            0.1 * g.standard_normal(sh) for sh in mlp.shapes(f_in, hidden, f_out)]


def test_gelu_matches_math_erf_and_its_derivative():
    xs = np.linspace(-6, 6, 121)
    want = np.array([0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in xs])
    np.testing.assert_allclose(mlp.gelu(xs), want, rtol=1e-15, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(xs), fd, rtol=1e-7, atol=1e-9)


def test_bce_is_negative_log_likelihood():
    g = np.random.Generator(np.random.PCG64(1))
    out = np.zeros((50, 3))
    out[:, 2] = g.standard_normal(50) * 4
    T = np.zeros((50, 3))
    T[:, 2] = g.integers(0, 2, 50)
    s = 1 / (1 + np.exp(-out[:, 2]))
    nll = -(T[:, 2] * np.log(s) + (1 - T[:, 2]) * np.log(1 - s))
    assert math.isclose(mlp.loss(out, T), float(np.mean(nll)), rel_tol=1e-12)


def test_gradients_match_finite_differences():
    f_in, hidden, f_out = 8, 16, 3
    params = _params(f_in, hidden, f_out, 3)
    g = np.random.Generator(np.random.PCG64(4))
    X = g.standard_normal((20, f_in))
    T = np.column_stack([g.standard_normal(20), g.uniform(-1, 1, 20), g.integers(0, 2, 20)])
    L, grads = mlp.loss_and_grad(params, X, T)
    flat = mlp.flatten(params)
    gflat = mlp.flatten(grads)
    h = 1e-6
    idx = g.choice(flat.size, 60, replace=False)
    for i in idx:
        fp = flat.copy(); fp[i] += h
        fm = flat.copy(); fm[i] -= h
        lp = mlp.loss(mlp.forward(mlp.unflatten(fp, f_in, hidden, f_out), X)[0], T)
        lm = mlp.loss(mlp.forward(mlp.unflatten(fm, f_in, hidden, f_out), X)[0], T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_flat_layout_round_trip():
    params = _params(8, 512, 3, 5)
    flat = mlp.flatten(params)
    assert flat.size == 8 * 512 + 512 + 2 * (512 * 512 + 512) + 3 * 512 + 3
    back = mlp.unflatten(flat)
    for a, b in zip(params, back):
        np.testing.assert_array_equal(a, b)


def test_bf16_round_ties_to_even_and_reduces_to_identity_network():
    # exactly representable, halfway cases (ties to even) and a value just above
    # a halfway point, against the definition: 8 significant bits
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0])
    np.testing.assert_array_equal(mlp.bf16_round(x), want)
    g = np.random.Generator(np.random.PCG64(5))
    v = g.standard_normal(1000)
    r = mlp.bf16_round(v)
    assert np.all(np.abs(r - v) <= 2.0 ** -8 * np.abs(v))                 # half an ulp of 8 bits
    # with the identity the rounded network is the FP64 network
    P = [g.standard_normal(sh) * 0.1 for sh in mlp.shapes(4, 16, 3)]
    X = g.standard_normal((7, 4))
    T = np.column_stack([g.standard_normal(7), g.standard_normal(7), g.integers(0, 2, 7)])
    L0, g0 = mlp.loss_and_grad(P, X, T)
    L1, g1 = mlp.loss_and_grad(P, X, T, round_act=lambda a: a)
    assert L0 == L1 and all(np.array_equal(a, b) for a, b in zip(g0, g1))
