"""Seeded input generators shared by the oracle tests and the GPU parity
tests.  They draw arrays with numpy's generator and hold none of the
simulation's arithmetic."""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def random_params(P, n_rows=1, seed=0, scale=0.3):
    """Parameter rows with a spread of magnitudes (float32)."""
    g = rng(seed)
    return (g.standard_normal((n_rows, P)) * scale).astype(np.float32)


def random_obs(D, seed=0, density=0.12):
    """A 0/1 patch with a trailing energy-like scalar block (float64)."""
    g = rng(seed)
    x = (g.random(D) < density).astype(np.float64)
    x[-1] = g.random()
    return x


def random_words(n, seed=0):
    return rng(seed).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
