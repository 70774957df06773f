"""Seeded initial parameters of the candidate-proposal network (an input, not the method).

Glorot-uniform weights and zero biases, packed as W1[9][64], b1[64], W2[64][64], b2[64],
W3[64][32], b3[32] (FP32), the layout of the library's parameter array.
"""
import numpy as np

SHAPES = [(9, 64), (64,), (64, 64), (64,), (64, 32), (32,)]


def mlp_init(seed: int = 1234) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for shp in SHAPES:
        if len(shp) == 2:
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            parts.append(rng.uniform(-lim, lim, size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts).astype(np.float32)
