"""The GPU EGO steps (Sec. II.A) against the FP64 oracle: maximin choice,
concentrated likelihood over a batch of theta vectors, kriging predictor,
MSE and expected improvement, and the whole loop on Branin's function.

Both sides are FP64; they differ in the order of the factorisation and of the
sums, which matters in proportion to the condition number of R.  Bars:
likelihoods 1e-9 relative where R is well conditioned (1e-6 where its
condition number reaches 1e11), predictions 1e-8 of the data scale, EI 1e-8 of
its maximum (FP64 route differences measured at 5e-13 on that model)."""
import os

import numpy as np
import pytest

from oracle import ego as oego
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, ego, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


def _data(n=40, d=3, seed=7):
    X = synth.unit_points(n, d, seed, 0)
    return X, np.sin(3.0 * X).sum(1) + X[:, 0] ** 2


def test_maximin_choice_matches(ctx):
    C = synth.lhs_candidates(40, 25, 4, seed=2)
    j, dmin = ego.lhs_maximin(ctx, C)
    jo, dmo = oego.maximin_select(C)
    assert j == jo
    assert np.allclose(dmin, dmo, rtol=1e-14, atol=0)


@pytest.mark.parametrize("lo,span,rtol", [(0.0, 2.0, 1e-9), (-1.0, 3.0, 1e-6)])
def test_likelihood_batch_matches(ctx, lo, span, rtol):
    # theta in [1, 100]: condition numbers up to 2.6e7, two FP64 routes agree to 4.5e-11;
    # theta down to 0.1: condition numbers up to 2.8e11, routes agree to 4.6e-8
    X, y = _data()
    th = 10.0 ** (lo + span * synth.theta_unit_draws(96, 3, 4, 0))
    got = ego.nll(ctx, X, y, th)
    ref = np.array([oego.nll(X, y, t) for t in th])
    assert np.all(np.isfinite(ref))
    assert np.allclose(got, ref, rtol=rtol, atol=rtol)
    assert int(np.argmin(got)) == int(np.argmin(ref))


def test_singular_correlation_gives_inf(ctx):
    X, y = _data()
    got = ego.nll(ctx, X, y, np.full((2, 3), 1e-9), nugget=0.0)   # R = all ones to 1e-9
    assert np.all(np.isinf(got))


def test_prediction_matches_over_two_chunks(ctx):
    X, y = _data()
    theta = np.array([2.0, 5.0, 1.0])
    gp = oego.fit(X, y, theta)
    C = synth.unit_points(40000, 3, 9, 1)                 # 32768 + a ragged second chunk
    f_min = float(y.min())
    ry, rs, rei = oego.predict(gp, C, f_min)
    with ego.Kriging(ctx, X, y, theta) as k:
        assert k.mu == pytest.approx(gp["mu"], rel=1e-10)
        assert k.sigma2 == pytest.approx(gp["sigma2"], rel=1e-9)
        gy, gs, gei = k.predict(C, f_min)
    scale = np.abs(y).max()
    assert np.abs(gy - ry).max() <= 1e-8 * scale
    assert np.abs(gs - rs).max() <= 1e-8 * scale
    assert np.abs(gei - rei).max() <= 1e-8 * rei.max()
    assert int(np.argmax(gei)) == int(np.argmax(rei))


def test_ego_on_branin(ctx):
    C = synth.lhs_candidates(50, 21, 2, seed=3)
    j, _ = ego.lhs_maximin(ctx, C)
    X0 = C[j]
    draws = lambda it: [synth.theta_unit_draws(32, 2, 5 + it, r) for r in range(4)]
    cands = lambda it: (synth.unit_points(2000, 2, 6, 2 * it), synth.unit_points(2000, 2, 6, 2 * it + 1))
    X, y, hist = ego.ego(ctx, synth.branin01, X0, synth.branin01(X0), 19, draws, cands)
    Xo, yo, _ = oego.ego(synth.branin01, X0, synth.branin01(X0), 19, draws, cands)
    print("GPU best", y.min(), "oracle best", yo.min())
    assert y.min() <= 0.397887 + 0.01
    # the first proposals coincide with the oracle's
    assert np.allclose(X[21:26], Xo[21:26], atol=1e-12)
