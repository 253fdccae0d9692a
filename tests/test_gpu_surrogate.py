"""Surrogate MLP on the GPU against the FP64 oracle MLP.

The GPU multiplies BF16 weights and BF16 activations with FP32 accumulation;
the oracle runs in FP64 at the same BF16-rounded weights and inputs, so the
remaining difference is the BF16 rounding of the activations and of dz between
layers (~2^-9 relative each, partly averaging out over the batch): measured
gradient errors are <= 1.1e-3 in norm per layer (bound 1e-2) with cosine
>= 0.999999 (bound 0.9999); the 24-step training loss curve agrees to ~1e-4
(bound 1 %)."""
import os

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1603_09493_gb300 import _lib as L
from paper_1603_09493_gb300 import api, synth

pytestmark = pytest.mark.gpu

SIZES = [16, 256, 256, 256, 256, 2]
CFG = (16, 256, 4, 2)


def bf16_round(x):
    x = np.asarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def dataset(N, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, size=(N, 16)).astype(np.float32)
    y0 = (X[:, 0] + 0.7 * X[:, 1] - 0.4 * X[:, 2] + 0.3 * X[:, 12] > 0.1).astype(np.float32)
    y1 = ((X[:, 3] * X[:, 4] > 0.1) & (X[:, 13] > -0.5)).astype(np.float32)
    return X, np.stack([y0, y1], 1)


@pytest.fixture(scope="module")
def ctx():
    if not os.path.exists(L.LIB_PATH):
        from paper_1603_09493_gb300 import build
        build.build()
    c = api.Context(0)
    yield c
    c.close()


def test_gradient_matches_oracle(ctx):
    params = synth.mlp_init_params(SIZES, seed=3)
    sur = ctx.surrogate(CFG, params)
    X, Y = dataset(1000, 1)                     # 1000 rows: padded to 1024 inside
    g, loss = sur.grad(X, Y)
    P = synth.unflatten_params(bf16_round(params), SIZES)
    logits, cache = omlp.forward(P, bf16_round(X).astype(np.float64))
    ref_loss = omlp.loss(logits, Y)
    grads = omlp.backward(P, cache, logits, Y)
    gref = synth.flatten_params(grads)
    assert abs(loss - ref_loss) <= 1e-2 * abs(ref_loss)
    off = 0
    for (W, b) in grads:
        for part in (W.ravel(), b.ravel()):
            gg = g[off:off + part.size].astype(np.float64)
            off += part.size
            if np.linalg.norm(part) < 1e-12:
                continue
            rel = np.linalg.norm(gg - part) / np.linalg.norm(part)
            cos = gg @ part / (np.linalg.norm(gg) * np.linalg.norm(part))
            print(f"size {part.size}: rel {rel:.3e} cos {cos:.6f}")
            assert rel <= 1e-2 and cos >= 0.9999
    assert off == gref.size == sur.P
    sur.destroy()


def test_training_matches_oracle_and_checkpoint(ctx, tmp_path):
    params = synth.mlp_init_params(SIZES, seed=5)
    X, Y = dataset(2048, 2)
    sur = ctx.surrogate(CFG, params)
    curve = sur.train(X, Y, epochs=3, batch=256, lr=1e-3, weight_decay=1e-4)
    P0 = synth.unflatten_params(bf16_round(params), SIZES)
    _, ref_curve = omlp.train(P0, bf16_round(X).astype(np.float64), Y.astype(np.float64), epochs=3, batch=256,
                              lr=1e-3, wd=1e-4)
    ref_curve = np.array(ref_curve)
    print("gpu", curve[[0, 5, 10, 23]], "oracle", ref_curve[[0, 5, 10, 23]])
    assert curve.shape == ref_curve.shape
    assert np.all(np.abs(curve - ref_curve) <= 0.01 * ref_curve)
    assert curve[-1] < 0.8 * curve[0]
    # inference at the trained weights against the oracle forward
    Xt, _ = dataset(3000, 9)
    pg = sur.infer(Xt)
    Pt = synth.unflatten_params(bf16_round(sur.params()), SIZES)
    lo, _ = omlp.forward(Pt, bf16_round(Xt).astype(np.float64))
    assert np.abs(pg - omlp.sigmoid(lo)).max() <= 0.02
    # checkpoint round trip into a fresh surrogate
    path = str(tmp_path / "sur.bin")
    sur.save(path)
    other = ctx.surrogate(CFG, np.zeros(sur.P, np.float32))
    other.load(path)
    assert np.array_equal(other.params(), sur.params())
    assert np.array_equal(other.infer(Xt), pg)
    sur.destroy()
    other.destroy()


def test_trained_surrogate_beats_prevalence(ctx):
    X, Y = dataset(8192, 4)
    Xt, Yt = dataset(4096, 5)
    sur = ctx.surrogate(CFG, synth.mlp_init_params(SIZES, seed=7))
    sur.train(X, Y, epochs=8, batch=512, lr=2e-3, weight_decay=1e-4)
    p = np.clip(sur.infer(Xt), 1e-6, 1 - 1e-6)
    bce = -np.mean(Yt * np.log(p) + (1 - Yt) * np.log(1 - p))
    prev = Y.mean(axis=0, keepdims=True)
    bce0 = -np.mean(Yt * np.log(prev) + (1 - Yt) * np.log(1 - prev))
    acc = np.mean((p > 0.5) == (Yt > 0.5))
    print(f"bce {bce:.3f} vs constant {bce0:.3f}, accuracy {acc:.3f}")
    assert bce < 0.5 * bce0 and acc > 0.9
    sur.destroy()


def test_screened_rates_match_oracle(ctx):
    # per-design means over jitter samples (Sec. II.C error rates) against the FP64 oracle at the
    # BF16-rounded weights and inputs; the bound is that of single-sample inference, 0.02
    params = synth.mlp_init_params(SIZES, seed=11)
    sur = ctx.surrogate(CFG, params)
    Pt = synth.unflatten_params(bf16_round(sur.params()), SIZES)
    for D, J in ((37, 7), (129, 1021)):                      # ragged; 131709 rows over three 65536-row chunks
        X, _ = dataset(D * J, 20 + J)
        R = sur.screen(X, D, J)
        ref = omlp.screened_ber(Pt, bf16_round(X).astype(np.float64), D, J)
        err = np.abs(R - ref).max()
        print(f"screen D={D} J={J}: max |d rate| {err:.2e}")
        assert R.shape == (D, 2) and err <= 0.02
        assert np.array_equal(sur.screen(X, D, J), R)          # fixed summation order
    # one sample per design: the rates are 1 - p and p of inference
    X, _ = dataset(300, 31)
    R, P = sur.screen(X, 300, 1), sur.infer(X).astype(np.float64)
    assert np.abs(R[:, 0] - (1.0 - P[:, 0])).max() <= 1e-6 and np.abs(R[:, 1] - P[:, 1]).max() <= 1e-6
    # device inputs give the host result
    import torch
    Xd = torch.from_numpy(X).cuda()
    assert np.array_equal(sur.screen(Xd, 300, 1).cpu().numpy(), R)
    sur.destroy()


def test_screened_rate_keeps_its_tail(ctx):
    # a constant network with output biases (40, -30): every logit is exactly the bias, and the write
    # error rate sigmoid(-40) = 4.2e-18 survives (1 - sigmoid(40) would round to 0 in any precision)
    flat = np.zeros_like(synth.mlp_init_params(SIZES, seed=0))
    flat[-2:] = [40.0, -30.0]
    sur = ctx.surrogate(CFG, flat)
    X, _ = dataset(5 * 9, 3)
    R = sur.screen(X, 5, 9)
    assert np.all(np.abs(R[:, 0] / (1.0 / (1.0 + np.exp(40.0))) - 1.0) <= 1e-12)
    assert np.all(np.abs(R[:, 1] / (1.0 / (1.0 + np.exp(30.0))) - 1.0) <= 1e-12)
    sur.destroy()


def test_screen_rejects_bad_arguments(ctx):
    sur = ctx.surrogate(CFG, synth.mlp_init_params(SIZES, seed=0))
    X, _ = dataset(8, 1)
    R = np.zeros((8, 2))
    assert ctx.lib.bpm_surrogate_screen(ctx.h, sur.sid, L.ptr(X), 0, 8, L.ptr(R), 0) == L.BPM_ERR_ARG
    assert ctx.lib.bpm_surrogate_screen(ctx.h, sur.sid, L.ptr(X), 8, 0, L.ptr(R), 0) == L.BPM_ERR_ARG
    assert ctx.lib.bpm_surrogate_screen(ctx.h, sur.sid + 99, L.ptr(X), 1, 8, L.ptr(R), 0) == L.BPM_ERR_ARG
    with pytest.raises(ValueError):
        sur.screen(X, 3, 3)
    sur.destroy()
