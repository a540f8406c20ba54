"""Brute-force IG on tiny item universes, straight from the definitions.

Every itemset b over the first L items (L <= 12) is enumerated and each
quantity of Section 3.1 is decided by its definition, by a route that differs
from the oracle's:

* b is in B^c (Eq. 1) iff some pair i < j has x_i AND x_j == b, or b equals a
  record of class c -- an existence check per b, instead of generating and
  deduplicating intersections;
* b is contained in x iff (b OR x) == x -- instead of the (b AND x) == b form of
  Eq. 6 that the oracle uses;
* |b| is counted with Python's bin(b).count("1").

Itemsets are Python ints (bit j = item j).  ``positions`` maps item j to a bit
position in the packed K-word layout, so the same brute force also covers
items that straddle a word boundary.
"""
from __future__ import annotations

import numpy as np


def pack(itemsets, positions, K):
    """Python-int itemsets over items 0..L-1 -> uint64[n, K] rows."""
    out = np.zeros((len(itemsets), K), dtype=np.uint64)
    for r, s in enumerate(itemsets):
        for j, pos in enumerate(positions):
            if (s >> j) & 1:
                out[r, pos // 64] |= np.uint64(1) << np.uint64(pos % 64)
    return out


def contains(x: int, b: int) -> bool:
    return (b | x) == x


def in_candidates(b: int, X) -> bool:
    if b == 0:
        return False
    if any(x == b for x in X):
        return True
    return any(X[i] & X[j] == b
               for i in range(len(X)) for j in range(i + 1, len(X)))


def fit(X_attack, X_normal, L):
    """Returns {cls: (B, P, f, S)} with B, P sorted lists of ints."""
    out = {}
    for cls, X, Y in ((1, X_attack, X_normal), (0, X_normal, X_attack)):
        B = [b for b in range(1, 1 << L) if in_candidates(b, X)]
        P = [b for b in B if not any(contains(y, b) for y in Y)]
        f = [sum(1 for x in X if contains(x, b)) for b in P]
        S = [fi * bin(b).count("1") ** 2 for fi, b in zip(f, P)]
        out[cls] = (B, P, f, S)
    return out


def evidence(P, S, t):
    return sum(s for b, s in zip(P, S) if contains(t, b))


def label(A, N, threshold=None):
    if A == 0 and N == 0:
        return 1
    if A >= N:
        return 1
    if threshold is not None and N < threshold:
        return 1
    return 0
