"""Seeded initial weights of the warm-start network (random numbers only, no method arithmetic).

Layer shapes (row-major W[in][out] followed by b[out]), in this order:
  coupling MLP: 16 -> 128 -> 128 -> 18;  output MLP: 20 -> 256 -> 256 -> 6.
W ~ N(0, 1/in); the last layer of each MLP is scaled by 1e-2 so the untrained network adds almost
nothing to the isolated-wire currents.  Biases start at zero.
"""
import numpy as np

LAYERS = [(16, 128), (128, 128), (128, 18), (20, 256), (256, 256), (256, 6)]


def n_params() -> int:
    return sum(i * o + o for i, o in LAYERS)


def init_params(seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for li, (i, o) in enumerate(LAYERS):
        w = rng.standard_normal((i, o)) / np.sqrt(i)
        if li in (2, len(LAYERS) - 1):
            w *= 1e-2
        parts += [w.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)
