"""Training the learned warm start's network on the method's own solutions.

The network (uoi_ws_* in include/uoi.h) predicts the converged ADMM state of
every (bootstrap, lambda, equation, feature) row from statistics that exist
before any iteration.  Its training rows come from uoi_ws_dataset: path-warm
FP64 ADMM solutions of synthetic problems shaped like the workload, drawn with
seeds disjoint from the workloads' data seeds (1000 + workload id), so a fit
of a workload never sees its own solutions.  The trained weights are saved to
a file that a fit reads through uoi_params.mlp_weights_path.
"""
from __future__ import annotations

import numpy as np

from . import native, synth

TRAIN_SEED_BASE = 90000          # problems for training rows: 90000 + i (workloads use 1001..1005)


def _block_weights(m, block_len, B, g):
    """Multiplicities of B block bootstraps of the m rows (blocks of block_len)."""
    L = max(int(block_len), 1)
    units = -(-m // L)
    w = np.zeros((B, m), dtype=np.uint32)
    for k in range(B):
        for u in g.integers(0, units, size=units):
            w[k, u * L:min(m, (u + 1) * L)] += 1
    return w


def _grid(X, Y, q, ratio=1e-3):
    lmax = float(np.max(np.abs(X.T @ Y))) / X.shape[0]
    return lmax * ratio ** (np.arange(q) / max(q - 1, 1))


def var_training_rows(p, T, density, radius, block_len, q, problems=2, B=2, max_rows=4_000_000):
    """(features, targets) from VAR(1) series of p channels (Eq. 7-9: p LASSOs
    sharing the lagged design), one lambda grid of q points per series."""
    feats, targs = [], []
    for i in range(problems):
        seed = TRAIN_SEED_BASE + i
        S = synth.var_problem(p, T, density, radius, seed=seed).series
        X, Y = np.ascontiguousarray(S[:-1]), np.ascontiguousarray(S[1:])
        g = np.random.Generator(np.random.PCG64(seed))
        w = _block_weights(X.shape[0], block_len, B, g)
        F, Tt = native.ws_dataset(X, Y, w, _grid(X, Y, q))
        feats.append(F)
        targs.append(Tt)
    F, Tt = np.concatenate(feats), np.concatenate(targs)
    if F.shape[0] > max_rows:
        keep = np.random.Generator(np.random.PCG64(TRAIN_SEED_BASE)).choice(F.shape[0], max_rows, replace=False)
        F, Tt = F[np.sort(keep)], Tt[np.sort(keep)]
    return F, Tt


def lasso_training_rows(n, p, nnz, q, problems=24, B=8, sigma=0.5):
    """(features, targets) from UoI_LASSO problems of n rows and p features."""
    feats, targs = [], []
    for i in range(problems):
        seed = TRAIN_SEED_BASE + i
        d = synth.lasso_problem(n, p, nnz, seed=seed, sigma=sigma)
        g = np.random.Generator(np.random.PCG64(seed))
        w = _block_weights(n, 1, B, g)
        F, Tt = native.ws_dataset(d.X, d.y, w, _grid(d.X, d.y.reshape(-1, 1), q))
        feats.append(F)
        targs.append(Tt)
    return np.concatenate(feats), np.concatenate(targs)


def train(features, targets, path, epochs=6, batch=4096, lr=1e-3, seed=1):
    """Trains a fresh network on the rows and saves its weights to path.
    Returns (initial loss on the first batch, final epoch loss)."""
    m = native.WarmStartModel(seed=seed)
    try:
        L0, _ = m.loss_grad(features[:batch], targets[:batch])
        L1 = m.train(features, targets, epochs=epochs, batch=batch, lr=lr, seed=seed + 4)
        m.save(path)
    finally:
        m.close()
    return L0, L1
