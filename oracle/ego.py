"""Efficient global optimisation (EGO) as the paper's optimiser uses it
(Sec. II.A), plain FP64 (oracle; test infrastructure).

The paper runs Dakota's EGO (Jones, Schonlau, Welch, J. Global Optim. 13, 455
(1998)): an optimised Latin hypercube of at least ten points per design
parameter fills the design space, a Gaussian process describes the
evaluated designs, and the design of highest expected improvement is
evaluated next; the process is refitted after every evaluation.  It prints
no formulas.  Readings used (Jones et al.'s kriging model):

* optimised Latin hypercube: among T random Latin hypercubes, the one whose
  smallest pairwise distance is largest (maximin);
* correlation R(x, x') = exp(-sum_k theta_k (x_k - x'_k)^2) on the unit cube,
  plus a fixed nugget on the diagonal of the training matrix;
* constant mean and variance by generalised least squares,
      mu = 1'R^-1 y / 1'R^-1 1,   sigma2 = (y - mu 1)' R^-1 (y - mu 1) / n,
  and theta by minimising the concentrated negative log-likelihood
      nll(theta) = n ln sigma2 + ln det R
  over rounds of T candidate log10 theta vectors: round 0 spans the box
  [lo, hi]^d, round r the box around the best so far with half-width
  (hi - lo) / 2^(r+1), clipped to [lo, hi];
* predictor and mean squared error at x with r = R(x, X):
      yhat = mu + r' R^-1 (y - mu 1),
      s2 = sigma2 [1 - r' R^-1 r + (1 - 1' R^-1 r)^2 / 1' R^-1 1];
* expected improvement below f_min = min y:
      EI = (f_min - yhat) Phi(z) + s phi(z),  z = (f_min - yhat) / s  (EI = 0 at s = 0);
* the next design is the candidate of largest EI among N uniform points of the
  unit cube and N points in the box of half-width 0.05 around the best design.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def maximin_select(cands: np.ndarray):
    """cands [T][n][d] -> (index of the maximin design, min squared distance of each)."""
    T = cands.shape[0]
    dmin = np.empty(T)
    for t in range(T):
        X = cands[t]
        D = np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=-1)
        iu = np.triu_indices(X.shape[0], 1)
        dmin[t] = D[iu].min()
    return int(np.argmax(dmin)), dmin


def corr(A: np.ndarray, B: np.ndarray, theta: np.ndarray) -> np.ndarray:
    D = (A[:, None, :] - B[None, :, :]) ** 2
    return np.exp(-np.einsum("ijk,k->ij", D, theta))


def _gls(X, y, theta, nugget):
    n = X.shape[0]
    R = corr(X, X, theta) + nugget * np.eye(n)
    L = np.linalg.cholesky(R)
    one = np.ones(n)
    Ri_y = np.linalg.solve(R, y)
    Ri_1 = np.linalg.solve(R, one)
    mu = (one @ Ri_y) / (one @ Ri_1)
    res = y - mu
    sigma2 = (res @ np.linalg.solve(R, res)) / n
    logdet = 2.0 * np.sum(np.log(np.diag(L)))
    return R, mu, sigma2, logdet, Ri_1


def nll(X, y, theta, nugget=1e-10) -> float:
    try:
        _, _, sigma2, logdet, _ = _gls(X, y, theta, nugget)
    except np.linalg.LinAlgError:
        return math.inf
    return X.shape[0] * math.log(sigma2) + logdet


def theta_search(X, y, draws, lo=-3.0, hi=2.0, nugget=1e-10):
    """draws: list of [T][d] unit uniforms, one per round.  Returns (theta, nll, all nll)."""
    best_c, best_v, allv = None, math.inf, []
    for r, U in enumerate(draws):
        if r == 0:
            a, b = np.full(U.shape[1], lo), np.full(U.shape[1], hi)
        else:
            h = (hi - lo) / 2.0 ** (r + 1)
            a, b = np.maximum(best_c - h, lo), np.minimum(best_c + h, hi)
        C = a + (b - a) * U
        for c in C:
            v = nll(X, y, 10.0 ** c, nugget)
            allv.append(v)
            if v < best_v:
                best_c, best_v = c, v
    return 10.0 ** best_c, best_v, np.array(allv)


def fit(X, y, theta, nugget=1e-10) -> dict:
    R, mu, sigma2, logdet, Ri_1 = _gls(X, y, theta, nugget)
    return dict(X=X, y=y, theta=theta, R=R, mu=mu, sigma2=sigma2, one_Ri_1=float(np.sum(Ri_1)),
                a=np.linalg.solve(R, y - mu))


def predict(gp: dict, C: np.ndarray, f_min: float):
    r = corr(C, gp["X"], gp["theta"])                   # [N][n]
    yhat = gp["mu"] + r @ gp["a"]
    Ri_r = np.linalg.solve(gp["R"], r.T)                 # [n][N]
    q = np.sum(r.T * Ri_r, axis=0)
    p = np.sum(Ri_r, axis=0)
    s2 = gp["sigma2"] * (1.0 - q + (1.0 - p) ** 2 / gp["one_Ri_1"])
    s = np.sqrt(np.maximum(s2, 0.0))
    ei = np.zeros_like(yhat)
    pos = s > 0
    z = (f_min - yhat[pos]) / s[pos]
    Phi = 0.5 * (1.0 + erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    ei[pos] = (f_min - yhat[pos]) * Phi + s[pos] * phi
    ei[~pos] = np.maximum(f_min - yhat[~pos], 0.0)
    return yhat, s, ei


def candidates(X, y, U_global, U_local, half=0.05):
    """The EI search set: uniform points plus points in the box around the best design."""
    best = X[int(np.argmin(y))]
    lo = np.clip(best - half, 0.0, 1.0)
    hi = np.clip(best + half, 0.0, 1.0)
    return np.concatenate([U_global, lo + (hi - lo) * U_local])


def ego(f, X0, y0, iters, draws_fn, cand_fn, nugget=1e-10):
    """draws_fn(it) -> list of theta-search unit draws; cand_fn(it) -> (U_global, U_local).
    Returns X, y and the per-iteration (theta, max EI)."""
    X, y, hist = np.array(X0, float), np.array(y0, float), []
    for it in range(iters):
        theta, _, _ = theta_search(X, y, draws_fn(it), nugget=nugget)
        gp = fit(X, y, theta, nugget)
        C = candidates(X, y, *cand_fn(it))
        _, _, ei = predict(gp, C, float(y.min()))
        j = int(np.argmax(ei))
        hist.append((theta, float(ei[j])))
        xn = C[j:j + 1]
        X = np.concatenate([X, xn])
        y = np.concatenate([y, f(xn)])
    return X, y, hist
