"""Seeded initial parameters of the shift-predictor MLP.

Both the CUDA training kernels and the CPU oracle start from these values, so that
their trajectories can be compared step by step.  The values are draws of
``numpy.random.default_rng(seed)``: weights uniform in +-sqrt(6 / (fan_in +
fan_out)), biases zero, laid out in the flat order W1 (8 x H row-major), b1 (H),
W2 (H x H row-major), b2 (H), w3 (H), b3.
"""
from __future__ import annotations

import numpy as np

NFEAT = 8


def mlp_init(hidden: int = 32, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    H = hidden

    def uni(fan_in, fan_out, size):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size)

    parts = [uni(NFEAT, H, NFEAT * H), np.zeros(H), uni(H, H, H * H), np.zeros(H), uni(H, 1, H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float64)
