"""Checks of tolerance-stopped LASSO columns against the exact minimiser (test helper).

For a selection column (bootstrap weights w_k, response e, lambda_j) the oracle
polishes its own FP64 ADMM iterate into the exact minimiser beta_hat of Eq. 2
(1/(2 n_k) scaling) and certifies it.  A point z returned by the CUDA path is
then held to what the stopping rule of Eq. 5 guarantees, with no free
allowance:
  * its KKT residual kappa = dist(0, dF(z)), computed in FP64 from FP64 moments,
    is at most ||H|| eps_pri + eps_dual, plus eta times the terms whose
    arithmetic the form rounds (oracle.admm_stop_bound); eta = 0 for the plain
    FP64 form, ETA_MIXED for the mixed form;
  * ||z - beta_hat|| <= kappa / lambda_min(H) (strong convexity of Eq. 2);
  * its support equals beta_hat's outside the band that kappa leaves open
    (oracle.support_band); the features inside the band are counted.

ETA_MIXED bounds the relative accuracy of the mixed form's arithmetic on the
quantities the x-update sees: moments from the two-piece bf16 Gram (elementwise
error <= 2e-6 of the largest diagonal, tested), the FP32-accurate inverse and
the two-piece fp16 x-update (a few 1e-7 each).
"""
import numpy as np

import oracle

ETA_MIXED = 2e-6


def moments(X, Y, w):
    """X^T W X, X^T W Y and n_k with numpy's matmul (a library primitive)."""
    Xw = X * np.asarray(w, dtype=np.float64)[:, None]
    return Xw.T @ X, Xw.T @ Y, float(np.sum(w))


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


class Report:
    def __init__(self):
        self.columns = 0
        self.band = 0
        self.max_rel = 0.0
        self.max_ratio = 0.0          # kappa / stopping bound
        self.bands = {}               # (k, j, e) -> band mask (for family checks)

    def __repr__(self):
        return (f"columns {self.columns}, features in the band {self.band}, "
                f"max rel l2 to the minimiser {self.max_rel:.2e}, max kappa/bound {self.max_ratio:.3f}")


def check_column(G, b, nk, lam, z, z_start, eta, mu, H_norm, rep, rho=1.0, abs_tol=1e-6,
                 rel_tol=1e-6):
    """One column; returns the band mask.  z_start: the oracle's iterate to polish."""
    pol = oracle.kkt_polish(G, b, nk, lam, z_start)
    assert pol["certified"], "the oracle's polish was not certified"
    bh = pol["beta"]
    p = G.shape[0]
    kap = oracle.kkt_residual(G, b, nk, lam, z)
    bound = oracle.admm_stop_bound(H_norm, p, z, lam, rho, abs_tol, rel_tol, eta,
                                   float(np.linalg.norm(b)) / nk)
    assert kap <= bound, f"KKT residual {kap:.3e} above the stopping bound {bound:.3e} (lambda {lam:.3e})"
    slack = 1e-12 * max(1.0, float(np.linalg.norm(bh)))
    dist = float(np.linalg.norm(z - bh))
    assert dist <= kap / mu + slack, f"distance {dist:.3e} above kappa/mu {kap / mu:.3e}"
    band = oracle.support_band(bh, pol["grad"], lam, kap + slack, mu, H_norm)
    mism = ((z != 0) != (bh != 0)) & ~band
    assert not mism.any(), f"{int(mism.sum())} support bits differ outside the band (lambda {lam:.3e})"
    rep.columns += 1
    rep.band += int(band.sum())
    rep.max_rel = max(rep.max_rel, rel_l2(z, bh))
    rep.max_ratio = max(rep.max_ratio, kap / bound if bound > 0 else 0.0)
    return band


def check_batch(X, Y, weights, lam, z_gpu, z_ref, eta, ks=None, eqs=None, js=None, rep=None,
                centre=False, **stop):
    """Columns (k, j, e) of B x q x r x p iterates; z_ref[a, j, b] is the oracle's
    iterate of z_gpu[ks[a], j, eqs[b]].  weights: B x n (rows ks).  centre: the
    w-centred moments (the selection problem of a fit with an intercept).
    Returns the report; rep.bands[(k, j, e)] holds each column's band."""
    rep = rep or Report()
    Y = Y.reshape(X.shape[0], -1)
    B, q, r, p = z_gpu.shape
    ks = list(range(B)) if ks is None else list(ks)
    eqs = list(range(r)) if eqs is None else list(eqs)
    js = list(range(q)) if js is None else list(js)
    for a, k in enumerate(ks):
        w = np.asarray(weights[a], dtype=np.float64)
        if centre:
            nk = float(w.sum())
            xb = (w @ X) / nk
            yb = (w @ Y) / nk
            G, Bm, nk = moments(X - xb, Y - yb, w)
        else:
            G, Bm, nk = moments(X, Y, w)
        ev = np.linalg.eigvalsh(G / nk)
        mu, Hn = float(ev[0]), float(ev[-1])
        assert mu > 0
        for b, e in enumerate(eqs):
            for j in js:
                rep.bands[(k, j, e)] = check_column(G, Bm[:, e], nk, lam[j], z_gpu[k, j, e],
                                                    z_ref[a, j, b], eta, mu, Hn, rep, **stop)
    return rep


def check_residuals(X, Y, weights, lam, z_gpu, eta, rep=None, **stop):
    """The statement that needs no strong convexity: every column's KKT residual is
    within the stopping bound (for problems whose bootstrap Gram is singular, where
    the minimiser need not be unique and the stopping rule decides no support)."""
    rep = rep or Report()
    Y = Y.reshape(X.shape[0], -1)
    B, q, r, p = z_gpu.shape
    rho, abs_tol, rel_tol = stop.get("rho", 1.0), stop.get("abs_tol", 1e-6), stop.get("rel_tol", 1e-6)
    for k in range(B):
        G, Bm, nk = moments(X, Y, weights[k])
        Hn = float(np.linalg.eigvalsh(G / nk)[-1])
        for e in range(r):
            for j in range(q):
                z = z_gpu[k, j, e]
                kap = oracle.kkt_residual(G, Bm[:, e], nk, lam[j], z)
                bound = oracle.admm_stop_bound(Hn, p, z, lam[j], rho, abs_tol, rel_tol, eta,
                                               float(np.linalg.norm(Bm[:, e])) / nk)
                assert kap <= bound, f"KKT residual {kap:.3e} above the stopping bound {bound:.3e}"
                rep.columns += 1
                rep.max_ratio = max(rep.max_ratio, kap / bound if bound > 0 else 0.0)
    return rep
