"""Efficient global optimisation (Sec. II.A; Jones, Schonlau, Welch 1998) on the
GPU path: the maximin Latin-hypercube choice, the concentrated kriging
likelihood, the kriging fit and the expected-improvement search all run in
libbpmllg (bpm_lhs_maximin, bpm_gp_nll, bpm_gp_create, bpm_gp_predict); this
module marshals arrays and runs the loop.

Readings (the paper names the method and its parts, not their formulas):
* the initial design is the maximin choice among random Latin hypercubes;
* theta is searched in rounds of candidate log10 vectors, round 0 over the
  box [lo, hi]^d, round r in the box around the best so far with half-width
  (hi - lo) / 2^(r+1), clipped; the smallest nll wins;
* the next design maximises EI over uniform points of the unit cube plus
  points in the box of half-width 0.05 around the best design so far.
"""
from __future__ import annotations

from ctypes import byref, c_double, c_int32

import numpy as np

from . import _lib as L


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def lhs_maximin(ctx, cands):
    """cands [T][n][d] -> (index of the maximin design, smallest squared distances [T])."""
    c = _f64(cands)
    T, n, d = c.shape
    best = c_int32()
    dmin = np.zeros(T)
    L.check(ctx.lib.bpm_lhs_maximin(ctx.h, L.ptr(c), T, n, d, byref(best), L.ptr(dmin)))
    return best.value, dmin


def nll(ctx, X, y, thetas, nugget=1e-10):
    """Concentrated negative log-likelihood of every theta row (natural, > 0)."""
    X, y, th = _f64(X), _f64(y), _f64(thetas)
    out = np.zeros(th.shape[0])
    L.check(ctx.lib.bpm_gp_nll(ctx.h, L.ptr(X), L.ptr(y), X.shape[0], X.shape[1], L.ptr(th), th.shape[0],
                               float(nugget), L.ptr(out)))
    return out


class Kriging:
    """A kriging model held on the device (bpm_gp_create / predict / destroy)."""

    def __init__(self, ctx, X, y, theta, nugget=1e-10):
        self.ctx = ctx
        X, y, th = _f64(X), _f64(y), _f64(theta)
        gid = c_int32()
        ms = np.zeros(2)
        L.check(ctx.lib.bpm_gp_create(ctx.h, L.ptr(X), L.ptr(y), X.shape[0], X.shape[1], L.ptr(th), float(nugget),
                                      byref(gid), L.ptr(ms)))
        self.id = gid.value
        self.mu, self.sigma2 = float(ms[0]), float(ms[1])

    def predict(self, C, f_min):
        C = _f64(C)
        N = C.shape[0]
        yh, s, ei = np.zeros(N), np.zeros(N), np.zeros(N)
        L.check(self.ctx.lib.bpm_gp_predict(self.ctx.h, self.id, L.ptr(C), N, float(f_min), L.ptr(yh), L.ptr(s),
                                            L.ptr(ei)))
        return yh, s, ei

    def close(self):
        if self.id >= 0:
            L.check(self.ctx.lib.bpm_gp_destroy(self.ctx.h, self.id))
            self.id = -1

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def theta_search(ctx, X, y, draws, lo=-3.0, hi=2.0, nugget=1e-10):
    """draws: list of [T][d] unit uniforms, one per round -> (theta, nll)."""
    best, best_v = None, np.inf
    d = X.shape[1]
    for r, U in enumerate(draws):
        if r == 0:
            a, b = np.full(d, lo), np.full(d, hi)
        else:
            h = (hi - lo) / 2.0 ** (r + 1)
            a, b = np.maximum(best - h, lo), np.minimum(best + h, hi)
        cand = a + (b - a) * np.asarray(U)
        v = nll(ctx, X, y, 10.0 ** cand, nugget)
        j = int(np.argmin(v))
        if v[j] < best_v:
            best, best_v = cand[j], float(v[j])
    return 10.0 ** best, best_v


def search_set(X, y, U_global, U_local, half=0.05):
    b = X[int(np.argmin(y))]
    lo, hi = np.clip(b - half, 0.0, 1.0), np.clip(b + half, 0.0, 1.0)
    return np.concatenate([U_global, lo + (hi - lo) * U_local])


def ego(ctx, f, X0, y0, iters, draws_fn, cand_fn, nugget=1e-10):
    """Run `iters` EGO iterations from the evaluated designs (X0, y0); f maps
    designs [m][d] in the unit cube to objective values [m].  Returns X, y and
    per-iteration (theta, max EI)."""
    X, y, hist = _f64(X0), _f64(y0), []
    for it in range(iters):
        theta, _ = theta_search(ctx, X, y, draws_fn(it), nugget=nugget)
        C = search_set(X, y, *cand_fn(it))
        with Kriging(ctx, X, y, theta, nugget) as gp:
            _, _, ei = gp.predict(C, float(y.min()))
        j = int(np.argmax(ei))
        hist.append((theta, float(ei[j])))
        X = np.concatenate([X, C[j:j + 1]])
        y = np.concatenate([y, np.asarray(f(C[j:j + 1]), np.float64)])
    return X, y, hist
