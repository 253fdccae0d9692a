"""Surrogate MLP, plain FP64 (oracle; test infrastructure).

The paper screens designs with a Gaussian-process model inside efficient
global optimisation (Sec. II.A); the surrogate here is a small multilayer
perceptron that predicts, from design/head/jitter features, the probability
that the target island switches and that an adjacent-track island flips.

Definitions used (textbook):
* layers x -> W1 x + b1 -> GELU -> ... -> W_L h + b_L (logits), W_l of shape
  [out][in]; GELU(x) = x * Phi(x) = x/2 (1 + erf(x / sqrt 2));
* loss = mean over samples and outputs of the sigmoid binary cross-entropy
  with logits: softplus(z) - y z;
* screened error rates of a design (Sec. II.C: a write error is a target island
  that fails to switch; an adjacent-track error is a neighbouring island that
  flips): over the J jittered samples of the design, the mean of
  P(no switch) = sigmoid(-z_0) and of P(flip) = sigmoid(z_k), k >= 1;
* AdamW (Loshchilov & Hutter, decoupled weight decay), bias-corrected moments:
      m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
      p -= lr * ( m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + wd * p )
  with weight decay on the weight matrices only (biases: wd = 0).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def forward(params, X):
    """params = [(W1, b1), ..., (WL, bL)]; returns logits and the cache."""
    h = np.asarray(X, np.float64)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < L - 1 else z
    return h, cache


def loss(logits, Y):
    return float(np.mean(softplus(logits) - Y * logits))


def backward(params, cache, logits, Y):
    """Gradients of `loss` w.r.t. every (W, b)."""
    Bn, O = logits.shape
    dz = (sigmoid(logits) - Y) / (Bn * O)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h_in, z = cache[l]
        W, _ = params[l]
        if l < len(params) - 1:
            dz = dz * gelu_grad(z)
        grads[l] = (dz.T @ h_in, dz.sum(axis=0))
        dz = dz @ W
    return grads


def adamw_step(params, grads, state, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update in place; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        state["v"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    state["t"] += 1
    t = state["t"]
    c1, c2 = 1.0 - beta1 ** t, 1.0 - beta2 ** t
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for j, (p, g, decay) in enumerate(((W, gW, wd), (b, gb, 0.0))):
            m = beta1 * state["m"][l][j] + (1.0 - beta1) * g
            v = beta2 * state["v"][l][j] + (1.0 - beta2) * g * g
            state["m"][l][j], state["v"][l][j] = m, v
            out.append(p - lr * ((m / c1) / (np.sqrt(v / c2) + eps) + decay * p))
        new.append(tuple(out))
    return new


def train(params, X, Y, epochs, batch, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """Minibatches taken in the given sample order, every epoch; the last
    partial batch is used as is.  Returns new params and the per-step losses."""
    state: dict = {}
    losses = []
    N = X.shape[0]
    for _ in range(epochs):
        for s in range(0, N, batch):
            xb, yb = X[s:s + batch], Y[s:s + batch]
            logits, cache = forward(params, xb)
            losses.append(loss(logits, yb))
            grads = backward(params, cache, logits, yb)
            params = adamw_step(params, grads, state, lr, wd, beta1, beta2, eps)
    return params, losses


def screened_ber(params, X, n_designs, n_jitter):
    """Per-design error rates from the surrogate over jitter samples (Sec. II.C).

    X [n_designs * n_jitter][n_in], design-major (rows d*J .. d*J + J - 1 are
    the jitter samples of design d).  Returns [n_designs][n_out]: column 0 the
    mean over the samples of the probability that the target island does not
    switch, sigmoid(-z_0); columns k >= 1 the mean probability of output k,
    sigmoid(z_k)."""
    logits, _ = forward(params, X)
    z = logits.reshape(n_designs, n_jitter, -1).copy()
    z[:, :, 0] = -z[:, :, 0]
    return sigmoid_tail(z).mean(axis=1)


def sigmoid_tail(z):
    """1 / (1 + exp(-z)) with full relative precision on both tails: a small
    probability is exp(z) / (1 + exp(z)), never a difference of values near 1."""
    z = np.asarray(z, np.float64)
    e = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + e), e / (1.0 + e))
