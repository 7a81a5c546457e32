"""Seeded weights of the linear softmax policy (input generator only).

W has shape [28224, 18] (the 84x84x4 stack flattened as plane, row, column
by 18 actions), drawn uniformly from (-a, a) with a = 1/sqrt(28224) = 1/168
and rounded to bfloat16 (round to nearest even on the float32 bits).
Returned as the uint16 bit patterns.
"""
from __future__ import annotations

import numpy as np

K, ACTIONS = 28224, 18


def policy_weights(seed: int = 5) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=seed + 0x5EED))
    u = g.uniform(-1.0 / 168.0, 1.0 / 168.0, size=(K, ACTIONS)).astype(np.float32)
    bits = u.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)
