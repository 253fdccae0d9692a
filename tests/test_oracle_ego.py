"""Pins of the EGO oracle (Sec. II.A; Jones, Schonlau, Welch 1998).

* maximin selection equals a brute-force pair loop;
* the GLS mean and variance maximise the Gaussian likelihood at fixed theta
  (checked against a numerical optimiser on the full likelihood);
* the kriging predictor and MSE are the limit of plain Gaussian conditioning
  with a diffuse prior on the constant mean (independent linear algebra);
* the expected improvement equals the integral of max(f_min - Y, 0) against
  the predictive normal (quadrature);
* the process interpolates its training data;
* EGO reaches the global minimum of Branin's function (0.397887), the test
  problem of Jones et al., within 0.01 in 40 evaluations."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import ego
from paper_1603_09493_gb300 import synth


def test_maximin_matches_brute_force():
    C = synth.lhs_candidates(12, 9, 3, seed=2)
    j, dmin = ego.maximin_select(C)
    brute = [min(float(np.sum((C[t, a] - C[t, b]) ** 2)) for a in range(9) for b in range(a + 1, 9))
             for t in range(12)]
    assert np.allclose(dmin, brute, rtol=1e-14)
    assert j == int(np.argmax(brute))


def _data(n=14, d=2, seed=7):
    X = synth.unit_points(n, d, seed, 0)
    return X, synth.branin01(X) if d == 2 else np.sin(3 * X).sum(1)


def test_gls_maximises_the_likelihood():
    X, y = _data()
    theta = np.array([3.0, 8.0])
    gp = ego.fit(X, y, theta)
    R = gp["R"]
    n = len(y)
    sign, logdet = np.linalg.slogdet(R)

    def negll(v):
        mu, ls2 = v
        r = y - mu
        return n * ls2 + logdet + (r @ np.linalg.solve(R, r)) / math.exp(ls2)

    res = optimize.minimize(negll, x0=[0.0, 0.0], method="Nelder-Mead",
                            options=dict(xatol=1e-10, fatol=1e-12, maxiter=20000))
    assert res.x[0] == pytest.approx(gp["mu"], rel=1e-6, abs=1e-6)
    assert math.exp(res.x[1]) == pytest.approx(gp["sigma2"], rel=1e-6)
    assert ego.nll(X, y, theta) == pytest.approx(n * math.log(gp["sigma2"]) + logdet, rel=1e-12)


def test_predictor_is_the_diffuse_prior_limit():
    X, y = _data()
    theta = np.array([3.0, 8.0])
    gp = ego.fit(X, y, theta)
    C = synth.unit_points(5, 2, 9, 1)
    yhat, s, _ = ego.predict(gp, C, float(y.min()))
    s2 = gp["sigma2"]
    tau2 = 1e6 * s2
    K = s2 * gp["R"] + tau2 * np.ones((len(y), len(y)))
    for c, x in enumerate(C):
        k = s2 * ego.corr(x[None], X, theta)[0] + tau2
        w = np.linalg.solve(K, k)
        assert yhat[c] == pytest.approx(w @ y, rel=1e-5, abs=1e-5 * np.abs(y).max())
        assert s[c] ** 2 == pytest.approx(s2 + tau2 - w @ k, rel=1e-4)


def test_expected_improvement_is_the_integral():
    X, y = _data()
    gp = ego.fit(X, y, np.array([3.0, 8.0]))
    C = synth.unit_points(6, 2, 11, 2)
    f_min = float(y.min())
    yhat, s, ei = ego.predict(gp, C, f_min)
    for c in range(len(C)):
        pdf = lambda t: math.exp(-0.5 * ((t - yhat[c]) / s[c]) ** 2) / (s[c] * math.sqrt(2 * math.pi))
        val, _ = integrate.quad(lambda t: (f_min - t) * pdf(t), yhat[c] - 12 * s[c], f_min, limit=200)
        assert ei[c] == pytest.approx(max(val, 0.0), rel=1e-7, abs=1e-12)


def test_interpolates_training_points():
    X, y = _data()
    gp = ego.fit(X, y, np.array([3.0, 8.0]))
    yhat, s, ei = ego.predict(gp, X, float(y.min()))
    assert np.allclose(yhat, y, atol=1e-6 * np.abs(y).max())
    assert np.all(s < 1e-3 * math.sqrt(gp["sigma2"]))


def _branin_run(iters=19):
    C = synth.lhs_candidates(50, 21, 2, seed=3)
    j, _ = ego.maximin_select(C)
    X0 = C[j]
    draws = lambda it: [synth.theta_unit_draws(32, 2, 5 + it, r) for r in range(4)]
    cands = lambda it: (synth.unit_points(2000, 2, 6, 2 * it), synth.unit_points(2000, 2, 6, 2 * it + 1))
    return ego.ego(synth.branin01, X0, synth.branin01(X0), iters, draws, cands)


def test_ego_finds_branin_minimum():
    X, y, hist = _branin_run()
    print("best", y.min(), "after", len(y), "evaluations")
    assert len(y) <= 40
    assert y.min() <= 0.397887 + 0.01
