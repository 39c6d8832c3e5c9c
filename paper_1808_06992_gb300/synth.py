"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only -- none of the method's arithmetic.
Both the CUDA path and the FP64 oracle are fed from it.  The paper's own
datasets (synthetic, unpublished; Sec. IV) and the NHP recordings are not
available, so these recipes stand in for them:

* ``lasso_problem``: the linear model of Eq. 1, y = X beta + eps, with
  iid N(0,1) or Toeplitz-correlated rows (Sigma_ij = rho^|i-j|, drawn by the
  AR(1) recursion over columns), a sparse beta with random support, random
  signs and uniform magnitudes, and Gaussian noise given either as sigma or
  as a signal-to-noise ratio (sigma^2 = beta' Sigma beta / SNR).
* ``var_problem``: the VAR(1) model of Eq. 6 with a sparse transition matrix
  A (N(0,1) entries) rescaled to a target spectral radius (the stability
  condition of Sec. II-G), N(0, I) innovations and a dropped burn-in.

All draws use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class LassoProblem:
    X: np.ndarray          # n x p, row-major float64
    y: np.ndarray          # n
    beta: np.ndarray       # p, the true coefficients
    sigma: float


@dataclass
class VarProblem:
    series: np.ndarray     # N x p, time ascending
    A: np.ndarray          # p x p true transition matrix
    burn_in: int = 0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def lasso_problem(n: int, p: int, nnz: int, *, seed: int, mag=(1.0, 3.0), sigma=None,
                  snr=None, toeplitz_rho: float = 0.0, dtype=np.float64) -> LassoProblem:
    g = _rng(seed)
    if toeplitz_rho == 0.0:
        X = g.standard_normal((n, p))
    else:
        # AR(1) over columns: x_j = rho x_{j-1} + sqrt(1 - rho^2) e_j gives
        # unit variances and Corr(x_i, x_j) = rho^|i-j|.
        X = np.empty((n, p))
        X[:, 0] = g.standard_normal(n)
        c = np.sqrt(1.0 - toeplitz_rho ** 2)
        for j in range(1, p):
            X[:, j] = toeplitz_rho * X[:, j - 1] + c * g.standard_normal(n)
    beta = np.zeros(p)
    idx = g.choice(p, size=nnz, replace=False)
    beta[idx] = g.uniform(mag[0], mag[1], size=nnz) * g.choice([-1.0, 1.0], size=nnz)
    if sigma is None:
        if snr is None:
            raise ValueError("give sigma or snr")
        if toeplitz_rho == 0.0:
            sig2 = float(beta @ beta) / snr
        else:
            lag = np.abs(np.arange(p)[:, None] - np.arange(p)[None, :])
            sig2 = float(beta @ (toeplitz_rho ** lag) @ beta) / snr
        sigma = float(np.sqrt(sig2))
    y = X @ beta + sigma * g.standard_normal(n)
    return LassoProblem(np.ascontiguousarray(X, dtype=dtype), np.ascontiguousarray(y, dtype=dtype),
                        beta, float(sigma))


def var_problem(p: int, T: int, density: float, spectral_radius: float, *, seed: int,
                burn_in: int = 500) -> VarProblem:
    g = _rng(seed)
    nnz = max(1, int(round(density * p * p)))
    A = np.zeros(p * p)
    pos = g.choice(p * p, size=nnz, replace=False)
    A[pos] = g.standard_normal(nnz)
    A = A.reshape(p, p)
    rad = float(np.max(np.abs(np.linalg.eigvals(A))))
    if rad > 0:
        A *= spectral_radius / rad
    total = T + burn_in
    U = g.standard_normal((total, p))
    S = np.empty((total, p))
    S[0] = U[0]
    for t in range(1, total):
        S[t] = A @ S[t - 1] + U[t]
    return VarProblem(np.ascontiguousarray(S[burn_in:]), A, burn_in)


@dataclass
class VarDProblem:
    series: np.ndarray      # T x p, time ascending
    A: np.ndarray           # order x p x p, A[j-1] = A_j
    mu: np.ndarray          # p
    burn_in: int


def var_d_problem(p: int, T: int, order: int, density: float, spectral_radius: float, *, seed: int,
                  mu_scale: float = 1.0, burn_in: int = 500) -> VarDProblem:
    """X_t = mu + sum_j A_j X_{t-j} + U_t, U_t ~ N(0, I): each A_j sparse with
    N(0,1) entries at random positions, then A_j scaled by c^j so that the
    companion matrix has the requested spectral radius (its eigenvalues scale
    by exactly c); mu ~ mu_scale * N(0, I)."""
    g = _rng(seed)
    nnz = max(1, int(round(density * p * p)))
    A = np.zeros((order, p * p))
    for j in range(order):
        A[j, g.choice(p * p, size=nnz, replace=False)] = g.standard_normal(nnz)
    A = A.reshape(order, p, p)
    comp = np.zeros((order * p, order * p))
    comp[:p] = np.concatenate(list(A), axis=1)
    comp[p:, :-p] = np.eye((order - 1) * p)
    rad = float(np.max(np.abs(np.linalg.eigvals(comp))))
    if rad > 0:
        c = spectral_radius / rad
        A *= (c ** np.arange(1, order + 1))[:, None, None]
    mu = mu_scale * g.standard_normal(p)
    total = T + burn_in
    U = g.standard_normal((total, p))
    S = np.zeros((total, p))
    for t in range(total):
        S[t] = mu + U[t]
        for j in range(1, min(order, t) + 1):
            S[t] += A[j - 1] @ S[t - j]
    return VarDProblem(np.ascontiguousarray(S[burn_in:]), A, mu, burn_in)


# ----------------------------------------------------------------------------
# The five workloads (data seed = 1000 + workload number)
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    kind: str                      # "lasso" | "var" | "batch"
    B1: int
    B2: int
    q: int
    block_len: int = 0
    bagging: int = 0               # 0 median, 1 mean
    params: dict = field(default_factory=dict)


WORKLOADS = {
    1: Workload("lasso_200x50_B1_20_q16_B2_10", "lasso", 20, 10, 16,
                params=dict(n=200, p=50, nnz=10, sigma=0.5)),
    2: Workload("lasso_50000x2000_toeplitz_B1_48_q48_B2_48", "lasso", 48, 48, 48,
                params=dict(n=50000, p=2000, nnz=100, snr=5.0, mag=(0.5, 3.0), toeplitz_rho=0.5)),
    3: Workload("var1_p192_T5000_B1_30_q32_B2_30_block100", "var", 30, 30, 32, block_len=100,
                params=dict(p=192, T=5000, density=0.03, spectral_radius=0.9)),
    4: Workload("batch64_uneven_lasso_B1_24_q32_B2_24", "batch", 24, 24, 32,
                params=dict(count=64, n=(500, 20000), p=(100, 1500), sparsity=(0.02, 0.10),
                            sigma=1.0)),
    5: Workload("var1_p1000_T20000_B1_32_q40_B2_32_block200", "var", 32, 32, 40, block_len=200,
                params=dict(p=1000, T=20000, density=0.01, spectral_radius=0.95)),
}


def workload_data(wid: int, scale: dict | None = None):
    """Inputs of workload ``wid`` (optionally with overridden sizes for tests)."""
    w = WORKLOADS[wid]
    prm = dict(w.params)
    if scale:
        prm.update(scale)
    seed = 1000 + wid
    if w.kind == "lasso":
        return lasso_problem(prm["n"], prm["p"], prm["nnz"], seed=seed, mag=prm.get("mag", (1.0, 3.0)),
                             sigma=prm.get("sigma"), snr=prm.get("snr"),
                             toeplitz_rho=prm.get("toeplitz_rho", 0.0))
    if w.kind == "var":
        return var_problem(prm["p"], prm["T"], prm["density"], prm["spectral_radius"], seed=seed)
    if w.kind == "batch":
        g = _rng(seed)
        count = prm["count"]
        ns = g.integers(prm["n"][0], prm["n"][1] + 1, size=count)
        ps = g.integers(prm["p"][0], prm["p"][1] + 1, size=count)
        sp = g.uniform(prm["sparsity"][0], prm["sparsity"][1], size=count)
        probs = []
        for i in range(count):
            nnz = max(1, int(round(sp[i] * ps[i])))
            probs.append(lasso_problem(int(ns[i]), int(ps[i]), nnz, seed=seed * 1000 + i,
                                       sigma=prm["sigma"]))
        return probs
    raise ValueError(w.kind)
