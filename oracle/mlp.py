"""FP64 reference of the warm-start MLP -- TEST INFRASTRUCTURE.

A plain numpy restatement of the network the CUDA library trains, used only to
check the library's forward pass and gradients.  Pinned by
tests/test_oracle_mlp.py (finite differences, GELU against math.erf, BCE
identity).

Network: x (F_IN) -> [W_l h + b_l, GELU] x 3 hidden layers of width H -> 3 outputs
(scaled z, scaled u, active logit).  GELU is the exact form 0.5 x (1 + erf(x/sqrt 2)).
Loss per row: (o0 - t0)^2 + (o1 - t1)^2 + softplus(o2) - t2 o2, averaged over rows.

Flat parameter layout (the library's documented format):
    W1 (H x F_IN), b1 (H), W2 (H x H), b2 (H), W3 (H x H), b3 (H), W4 (3 x H), b4 (3),
each matrix row-major [out][in].
"""
from __future__ import annotations

import math

import numpy as np

F_IN, HIDDEN, F_OUT = 8, 512, 3


def shapes(f_in=F_IN, hidden=HIDDEN, f_out=F_OUT):
    return [(hidden, f_in), (hidden,), (hidden, hidden), (hidden,), (hidden, hidden), (hidden,),
            (f_out, hidden), (f_out,)]


def unflatten(flat, f_in=F_IN, hidden=HIDDEN, f_out=F_OUT):
    out, o = [], 0
    for sh in shapes(f_in, hidden, f_out):
        n = int(np.prod(sh))
        out.append(np.asarray(flat[o:o + n], dtype=np.float64).reshape(sh))
        o += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in params])


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def bf16_round(x):
    """Nearest BF16 value (ties to even) of each value taken to FP32 first: the
    rounding of a value the GPU holds in FP32 and stores as BF16."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(x):
    return x


def forward(params, X, round_act=_identity):
    """round_act is applied to each hidden activation h_l after the GELU (the
    values the GPU stores in BF16 for the next product); identity = FP64 network."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    a1 = X @ W1.T + b1
    h1 = round_act(gelu(a1))
    a2 = h1 @ W2.T + b2
    h2 = round_act(gelu(a2))
    a3 = h2 @ W3.T + b3
    h3 = round_act(gelu(a3))
    out = h3 @ W4.T + b4
    return out, (X, a1, h1, a2, h2, a3, h3)


def softplus(x):
    return np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))), np.log1p(np.exp(-np.abs(x))))


def loss(out, T):
    d0 = out[:, 0] - T[:, 0]
    d1 = out[:, 1] - T[:, 1]
    bce = softplus(out[:, 2]) - T[:, 2] * out[:, 2]
    return float(np.mean(d0 * d0 + d1 * d1 + bce))


def loss_and_grad(params, X, T, round_act=_identity):
    """Loss and gradient (same structure as params) by explicit backpropagation.
    round_act is also applied to each back-propagated da_l (stored in BF16 on the
    GPU); the gradient is that of the network with the rounding held fixed."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    out, (X, a1, h1, a2, h2, a3, h3) = forward(params, X, round_act)
    N = X.shape[0]
    L = loss(out, T)
    dout = np.empty_like(out)
    dout[:, 0] = 2.0 * (out[:, 0] - T[:, 0]) / N
    dout[:, 1] = 2.0 * (out[:, 1] - T[:, 1]) / N
    dout[:, 2] = (1.0 / (1.0 + np.exp(-out[:, 2])) - T[:, 2]) / N
    gW4 = dout.T @ h3
    gb4 = dout.sum(0)
    da3 = round_act((dout @ W4) * gelu_grad(a3))
    gW3 = da3.T @ h2
    gb3 = da3.sum(0)
    da2 = round_act((da3 @ W3) * gelu_grad(a2))
    gW2 = da2.T @ h1
    gb2 = da2.sum(0)
    da1 = round_act((da2 @ W2) * gelu_grad(a1))
    gW1 = da1.T @ X
    gb1 = da1.sum(0)
    return L, [gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4]
