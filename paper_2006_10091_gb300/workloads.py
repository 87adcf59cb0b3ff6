"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module only draws numbers and lays them out in slots; it holds none of
the homomorphic arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it.  The paper's data sets (MNIST 3-vs-8, the credit data
set, FEMNIST) are not available; these generators stand in for them with the
shapes the encrypted logistic-regression step is measured on.
"""
from __future__ import annotations

import math

import numpy as np


def uniform_slots(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """`count` float64 values uniform in [lo, hi)."""
    return np.random.default_rng(seed).uniform(lo, hi, count)


def int_poly(seed: int, n: int, bound: int) -> np.ndarray:
    """Integer plaintext coefficients uniform in [-bound, bound] (int64)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-bound, bound + 1, size=n, dtype=np.int64)


def residues(seed: int, primes, n: int, parts: int = 1) -> np.ndarray:
    """Uniform residues [parts][len(primes)][n] (uint64), limb t below primes[t]."""
    rng = np.random.default_rng(seed)
    out = np.empty((parts, len(primes), n), dtype=np.uint64)
    for t, q in enumerate(primes):
        out[:, t, :] = rng.integers(0, int(q), size=(parts, n), dtype=np.uint64)
    return out


class LRData:
    """Two-class data: X (n x d) with ~`zero_frac` zeros and other entries
    uniform in (0, 1]; labels +-1 from a planted Gaussian w* thresholded at
    the median score (balanced classes); initial weights uniform in
    [-0.5, 0.5]."""

    def __init__(self, seed: int, n_samples: int, n_features: int, zero_frac: float = 0.8):
        rng = np.random.default_rng(seed)
        x = rng.uniform(0.0, 1.0, (n_samples, n_features))
        x = np.where(x == 0.0, 1.0, x)  # (0, 1]
        keep = rng.uniform(0.0, 1.0, (n_samples, n_features)) >= zero_frac
        self.X = np.where(keep, x, 0.0)
        w_star = rng.normal(0.0, 1.0, n_features)
        score = self.X @ w_star
        self.y = np.where(score > np.median(score), 1.0, -1.0)
        self.w0 = rng.uniform(-0.5, 0.5, n_features)
        self.n, self.d = n_samples, n_features


def lr_layout(n_slots: int, g: int, n_features: int):
    """Interleaved slot layout used by the step: g samples per ciphertext,
    F = n_slots / g feature positions, slot g*f + s holds (sample s, feature
    f).  Returns F; raises if the features do not fit."""
    if g < 1 or (g & (g - 1)) or n_slots % g:
        raise ValueError("g must be a power of two dividing the slot count")
    F = n_slots // g
    if n_features > F:
        raise ValueError(f"{n_features} features do not fit {F} positions")
    return F


def pack_samples(X: np.ndarray, y: np.ndarray, n_slots: int, g: int) -> list[np.ndarray]:
    """Slot vectors z_k with slot g*f + s = y_i * x_{i,f} for the s-th sample
    of group k (zero padding for missing samples and features)."""
    n, d = X.shape
    F = lr_layout(n_slots, g, d)
    n_ct = math.ceil(n / g)
    out = []
    for k in range(n_ct):
        v = np.zeros(n_slots)
        for s in range(g):
            i = k * g + s
            if i >= n:
                break
            v[s:g * d:g] = y[i] * X[i]
        out.append(v)
    del F
    return out


def pack_weights(w: np.ndarray, n_slots: int, g: int) -> np.ndarray:
    """Slot vector with w_f in slots g*f + s for every s."""
    F = lr_layout(n_slots, g, len(w))
    v = np.zeros(n_slots)
    for s in range(g):
        v[s:g * len(w):g] = w
    del F
    return v


def shard_sizes(seed: int, k: int, lo: int = 512, hi: int = 8192) -> list[int]:
    """`k` shard sizes log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), k)]


def shard_levels(seed: int, k: int, lo: int = 2, hi: int = 8) -> list[int]:
    """`k` remaining levels uniform in {lo..hi}."""
    rng = np.random.default_rng(seed + 7919)
    return [int(v) for v in rng.integers(lo, hi + 1, k)]


def poisson_arrivals(seed: int, rate: float, count: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))
