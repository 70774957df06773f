"""FP64 reference of the candidate-proposal network -- TEST INFRASTRUCTURE ONLY.

Plain numpy: forward pass, masked softmax cross-entropy (softmax over the first
n_cand of 32 outputs) and the backward pass by the chain rule, for the packed
parameter layout W1[9][64], b1[64], W2[64][64], b2[64], W3[64][32], b3[32].
GELU is the erf form x * Phi(x).  An optional emulation of BF16 storage
(round-to-nearest-even of weights and layer inputs) mirrors where the tensor-core
path rounds, for comparing logits.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss, the
closed form log(n_cand) at zero weights, and the masking of slots >= n_cand.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

SHAPES = [(9, 64), (64,), (64, 64), (64,), (64, 32), (32,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in parts])


def bf16(x):
    """Round FP32 values to BF16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + special.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(p, X, emulate_bf16=False):
    """Logits (n, 32) and the intermediates."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    r = bf16 if emulate_bf16 else (lambda a: a)
    Z1 = r(X) @ r(W1) + b1
    H1 = gelu(Z1)
    Z2 = r(H1) @ r(W2) + b2
    H2 = gelu(Z2)
    Z3 = r(H2) @ r(W3) + b3
    return Z3, (X, Z1, H1, Z2, H2)


def masked_log_softmax(Z3, ncand):
    n = np.asarray(ncand)
    mask = np.arange(Z3.shape[1])[None, :] < n[:, None]
    Zm = np.where(mask, Z3, -np.inf)
    m = Zm.max(axis=1, keepdims=True)
    lse = m + np.log(np.exp(Zm - m).sum(axis=1, keepdims=True))
    return np.where(mask, Z3 - lse, -np.inf), mask


def loss_and_grad(p, X, label, ncand):
    """Mean cross-entropy over the samples and its gradient (packed)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Z3, (X, Z1, H1, Z2, H2) = forward(p, X)
    logp, mask = masked_log_softmax(Z3, ncand)
    n = X.shape[0]
    y = np.asarray(label)
    loss = -logp[np.arange(n), y].mean()
    P = np.where(mask, np.exp(logp), 0.0)
    dZ3 = P.copy()
    dZ3[np.arange(n), y] -= 1.0
    dZ3 /= n
    dW3 = H2.T @ dZ3
    db3 = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ W3.T) * gelu_grad(Z2)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * gelu_grad(Z1)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(axis=0)
    return float(loss), pack([dW1, db1, dW2, db2, dW3, db3])


def loss_only(p, X, label, ncand):
    Z3, _ = forward(p, X)
    logp, _ = masked_log_softmax(Z3, ncand)
    return float(-logp[np.arange(X.shape[0]), np.asarray(label)].mean())
