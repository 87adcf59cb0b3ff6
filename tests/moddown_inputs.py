"""Key-switch accumulators whose dropped part lifts next to 0 and next to the
dropped modulus, for the ModDown tests (oracle pins and GPU parity).

ModDown divides an accumulator over Q_l * P by P with rounding (and, merged
with the multiplication's rescale, P (d0, d1) + acc by P q_{l-1}): with D the
dropped modulus and h = (D - 1)/2, the coefficient X becomes
floor((X + h) / D).  The conversion behind it lifts (X + h) mod D from its
residues; a lift of 0, 1, 2, D - 2 or D - 1 is where a fixed-point count of
the multiples of D can go wrong.  These builders choose the integers X
themselves (Python integers) and return their residues, so that the expected
result is known exactly.  Evaluation form is taken with the oracle's
transform (the inputs never come from the CUDA path).
"""
from __future__ import annotations

import math
import random

import numpy as np

import oracle

BOUNDARY = (0, 1, 2, -2, -1)  # lifts of (X + h) mod D, taken mod D


def coefficient_integers(M: int, D: int, n: int, seed: int, reps: int = 4) -> list[int]:
    """n integers in [0, M) (D divides M): the first len(BOUNDARY) * reps have
    (X + h) mod D in BOUNDARY (spread over the polynomial), the rest uniform."""
    rng = random.Random(seed)
    h = (D - 1) // 2
    xs = [rng.randrange(M) for _ in range(n)]
    nb = min(n, len(BOUNDARY) * reps)
    for i in range(nb):
        pos = i * (n // nb)
        b = BOUNDARY[i % len(BOUNDARY)] % D
        xs[pos] = rng.randrange(M // D) * D + (b - h) % D
    return xs


def to_eval(o, coef_rows, prime_indices) -> np.ndarray:
    """Coefficient residues -> evaluation form, limb by limb (oracle NTT)."""
    return np.stack([oracle.ntt_r2(np.asarray(row, dtype=np.uint64), o.log_n, o.primes[t], o.roots[t])
                     for row, t in zip(coef_rows, prime_indices)])


def accumulator(o, level: int, seed: int, merged: bool = False):
    """(acc [2][level + alpha][N] evaluation form, d01 [2][level][N] or None,
    X [2][N] Python integers, D): acc's lift over Q_level * P (with P d01
    added when merged) is X."""
    q, L, alpha, n = o.primes, o.L, o.alpha, o.n
    tp = list(range(level)) + list(range(L, L + alpha))  # prime index of each accumulator limb
    M = math.prod(q[t] for t in tp)
    P = math.prod(q[L:L + alpha])
    D = P * q[level - 1] if merged else P
    rng = np.random.default_rng(seed)
    acc = np.empty((2, level + alpha, n), dtype=np.uint64)
    d01 = np.empty((2, level, n), dtype=np.uint64) if merged else None
    X = []
    for p in range(2):
        xs = coefficient_integers(M, D, n, seed * 2 + p)
        X.append(xs)
        dc = [rng.integers(0, q[t], n, dtype=np.uint64) for t in range(level)] if merged else None
        rows = []
        for i, t in enumerate(tp):
            m = q[t]
            r = [x % m for x in xs]
            if merged and t < level:  # acc = X - P d on the limbs of Q_level
                pm = P % m
                r = [(v - pm * int(dv)) % m for v, dv in zip(r, dc[t])]
            rows.append(r)
        acc[p] = to_eval(o, rows, tp)
        if merged:
            d01[p] = to_eval(o, dc, list(range(level)))
    return acc, d01, X, D


def expected_coef(X, D: int, primes) -> list[list[list[int]]]:
    """floor((X + h) / D) mod each prime, [2][len(primes)][N] (coefficient form)."""
    h = (D - 1) // 2
    return [[[((x + h) // D) % m for x in xs] for m in primes] for xs in X]
