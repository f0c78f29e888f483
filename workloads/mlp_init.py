"""Seeded initial parameters of the learned-pruning MLP (an input of the
training, like a circuit's angles): He-uniform weights and zero biases for the
16 -> 128 -> 128 -> 1 layout W1[16][128], b1, W2[128][128], b2, w3[128], b3."""
import numpy as np

N_PARAMS = 18817


def mlp_init_params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAMS)
    p[0:2048] = rng.uniform(-1, 1, 2048) * np.sqrt(6.0 / 16)
    p[2176:18560] = rng.uniform(-1, 1, 128 * 128) * np.sqrt(6.0 / 128)
    p[18688:18816] = rng.uniform(-1, 1, 128) * np.sqrt(6.0 / 128)
    return p.astype(np.float32)
