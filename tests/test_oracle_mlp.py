"""Pins for the FP64 reference of the proposal network: central finite differences,
the closed-form loss at zero weights, masking and the BF16 rounding rule."""
import math

import numpy as np

from oracle import mlp
from synth.mlp_init import mlp_init


def data(n=24, seed=0):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.uniform(-1, 1, (n, 8)), np.ones((n, 1))], axis=1)
    nc = rng.integers(2, 33, n)
    y = np.array([rng.integers(0, k) for k in nc])
    X[:, 7] = nc / 32.0
    return X, y, nc


def test_gradient_matches_central_differences():
    X, y, nc = data()
    p = mlp_init(3).astype(np.float64) + np.random.default_rng(1).normal(0, 0.05, mlp.N_PARAMS)
    loss, g = mlp.loss_and_grad(p, X, y, nc)
    assert abs(loss - mlp.loss_only(p, X, y, nc)) < 1e-14
    rng = np.random.default_rng(2)
    for i in rng.choice(mlp.N_PARAMS, 200, replace=False):
        e = np.zeros(mlp.N_PARAMS)
        h = 1e-6
        e[i] = h
        fd = (mlp.loss_only(p + e, X, y, nc) - mlp.loss_only(p - e, X, y, nc)) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_weights_give_uniform_softmax():
    X, y, nc = data()
    loss, g = mlp.loss_and_grad(np.zeros(mlp.N_PARAMS), X, y, nc)
    assert abs(loss - np.mean(np.log(nc))) < 1e-12


def test_masked_slots_get_no_probability_or_gradient():
    X, y, nc = data()
    p = mlp_init(4).astype(np.float64)
    Z3, _ = mlp.forward(p, X)
    logp, mask = mlp.masked_log_softmax(Z3, nc)
    P = np.where(mask, np.exp(logp), 0.0)
    assert np.allclose(P.sum(axis=1), 1.0)
    assert np.all(P[~mask] == 0.0)
    # logits of masked slots do not influence the loss: b3 gradient is zero beyond max(nc)
    X2, y2 = X[nc < 20], y[nc < 20]
    _, g = mlp.loss_and_grad(p, X2, y2, nc[nc < 20])
    b3 = mlp.unpack(g)[5]
    assert np.all(b3[19:] == 0.0)


def test_bf16_rounding_rule():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, 3.1415926, -2.5e-3], dtype=np.float32)
    r = mlp.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # halfway between 1 and 1 + 2^-7: ties to even
    assert r[2] == 1.0 + 2 ** -7              # nearest representable (spacing 2^-7 near 1)
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)
