"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds none of the solver's arithmetic: only random vectors and matrices drawn
from numpy's PCG64 with fixed seeds.  The benchmark's own system (A, b) comes
from each side's generator, not from here.
"""
import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def vectors(n: int, k: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """n x k fp64 matrix (Fortran order), entries uniform in (-scale, scale)."""
    return np.asfortranarray(rng(seed).uniform(-scale, scale, size=(n, k)))


def doubles_spanning(count: int, seed: int, lo_exp: int, hi_exp: int) -> np.ndarray:
    """Signed fp64 values with log-uniform magnitudes in [2^lo_exp, 2^hi_exp)."""
    g = rng(seed)
    mag = np.exp2(g.uniform(lo_exp, hi_exp, size=count))
    return mag * np.where(g.random(count) < 0.5, -1.0, 1.0)
