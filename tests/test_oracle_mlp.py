"""Pins of the oracle MLP: finite-difference gradients, GELU/BCE closed forms,
the closed form of the first AdamW step, the screened error rates of a
constant network."""
import math

import numpy as np

from oracle import mlp


def _params(sizes, seed):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((o, i)) / math.sqrt(i), 0.1 * rng.standard_normal(o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_gelu_and_bce_closed_forms():
    assert mlp.gelu(np.array(0.0)) == 0.0
    # GELU(1) = Phi(1) = 0.8413447460685429
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array(8.0)) - 8.0) < 1e-12 and abs(mlp.gelu(np.array(-8.0))) < 1e-12
    z = np.zeros((3, 2))
    assert abs(mlp.loss(z, np.ones((3, 2))) - math.log(2)) < 1e-15
    # large logits: loss -> |z| on the wrong side, 0 on the right side
    assert abs(mlp.loss(np.array([[40.0]]), np.array([[0.0]])) - 40.0) < 1e-12
    assert mlp.loss(np.array([[40.0]]), np.array([[1.0]])) < 1e-15


def test_gradients_match_central_differences():
    sizes = [16, 12, 10, 8, 2]
    params = _params(sizes, 0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 16))
    Y = (rng.random((7, 2)) < 0.4).astype(float)
    logits, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, logits, Y)
    eps = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gf = g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = mlp.loss(mlp.forward(params, X)[0], Y)
                flat[idx] = old - eps
                lm = mlp.loss(mlp.forward(params, X)[0], Y)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gf[idx]) < 1e-7 * max(1.0, abs(fd)), (l, idx, fd, gf[idx])


def test_first_adamw_step_closed_form():
    params = _params([4, 3, 2], 2)
    grads = [(np.full_like(W, 0.5), np.full_like(b, -2.0)) for W, b in params]
    lr, wd, eps = 1e-3, 0.01, 1e-8
    new = mlp.adamw_step(params, grads, {}, lr, wd, eps=eps)
    for (W, b), (W1, b1), (gW, gb) in zip(params, new, grads):
        # bias corrections cancel on step 1: update = g / (|g| + eps)
        assert np.allclose(W1, W - lr * (gW / (np.abs(gW) + eps) + wd * W), atol=1e-15)
        assert np.allclose(b1, b - lr * (gb / (np.abs(gb) + eps)), atol=1e-15)


def test_training_reduces_loss_on_a_separable_task():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((256, 16))
    Y = np.stack([(X[:, 0] + X[:, 1] > 0), (X[:, 2] > 0.5)], 1).astype(float)
    params = _params([16, 32, 32, 2], 4)
    _, losses = mlp.train(params, X, Y, epochs=20, batch=64, lr=3e-3, wd=1e-4)
    assert losses[-1] < 0.5 * losses[0]


def test_screened_ber_of_a_constant_network():
    # zero weights: every logit is its bias, so design error rates are closed forms
    sizes = [16, 8, 2]
    params = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(sizes[:-1], sizes[1:])]
    params[-1] = (np.zeros((2, 8)), np.array([2.0, -3.0]))
    X = np.random.default_rng(1).uniform(-1, 1, size=(5 * 3, 16))
    r = mlp.screened_ber(params, X, 5, 3)
    assert r.shape == (5, 2)
    assert np.allclose(r[:, 0], 1.0 / (1.0 + math.exp(2.0)), rtol=1e-15, atol=0)     # P(no switch) at z = 2
    assert np.allclose(r[:, 1], 1.0 / (1.0 + math.exp(3.0)), rtol=1e-15, atol=0)     # P(flip) at z = -3
    # a far-switching target: the write error rate keeps its relative precision (no 1 - p cancellation)
    params[-1] = (np.zeros((2, 8)), np.array([40.0, 0.0]))
    r = mlp.screened_ber(params, X, 5, 3)
    assert abs(r[0, 0] / math.exp(-40.0) - 1.0) < 1e-12 and r[0, 1] == 0.5


def test_screened_ber_is_a_per_design_mean():
    sizes = [16, 12, 2]
    params = _params(sizes, 3)
    D, J = 4, 6
    X = np.random.default_rng(2).uniform(-1, 1, size=(D * J, 16))
    r = mlp.screened_ber(params, X, D, J)
    # brute force, one sample at a time
    for d in range(D):
        acc = np.zeros(2)
        for j in range(J):
            z, _ = mlp.forward(params, X[d * J + j][None])
            acc += [1.0 / (1.0 + math.exp(z[0, 0])), 1.0 / (1.0 + math.exp(-z[0, 1]))]
        assert np.allclose(r[d], acc / J, rtol=1e-13, atol=0)
    # the order of a design's samples does not matter; designs do not mix
    perm = np.concatenate([d * J + np.random.default_rng(d).permutation(J) for d in range(D)])
    assert np.allclose(mlp.screened_ber(params, X[perm], D, J), r, rtol=1e-13, atol=0)
    assert np.allclose(mlp.screened_ber(params, X[:J], 1, J), r[:1], rtol=1e-15, atol=0)
