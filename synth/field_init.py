"""Seeded initial parameters of the neural density field (data only: random numbers drawn once
and passed to both the oracle and the CUDA trainer).

Hidden and output weights are uniform in +-sqrt(6 / fan_in) (He et al. 2015, uniform form),
biases start at zero; packed as W1, b1, W2, b2, W3, b3, W4, b4, w5, b5 (row = output unit)."""
import numpy as np

WIDTH, DEPTH = 64, 4
N_PARAMS = DEPTH * (WIDTH * WIDTH + WIDTH) + WIDTH + 1


def field_init(seed: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lim = np.sqrt(6.0 / WIDTH)
    parts = []
    for _ in range(DEPTH):
        parts.append(rng.uniform(-lim, lim, size=WIDTH * WIDTH))
        parts.append(np.zeros(WIDTH))
    parts.append(rng.uniform(-lim, lim, size=WIDTH))
    parts.append(np.zeros(1))
    return np.concatenate(parts).astype(np.float32)
