"""The item index's pruning is exact, checked on the CPU by brute force.

The item-index form of the subset test (prune.cu, and its tensor-core
blocks) files every record under each item it holds and every pattern under
its key item -- the item of the pattern held by the fewest records, the
lowest such item on ties -- and tests a pattern only against the records of
its key item's group; a pattern with an item no record holds is inside no
record and is not tested at all.  A record containing p holds every item of
p, in particular its key item, so no containing pair is lost, and each pair
is met in exactly one group.  This test restates the filing in Python and
checks, on random packed itemsets, that the (pattern, record) pairs with
p inside r found through the index are exactly those of the full product,
with fewer tests executed.
"""
import numpy as np
import pytest


def items(row):
    out = []
    for w, word in enumerate(row):
        x = int(word)
        while x:
            b = (x & -x).bit_length() - 1
            out.append(64 * w + b)
            x &= x - 1
    return out


def contains(r, p):
    return all((int(rw) & int(pw)) == int(pw) for rw, pw in zip(r, p))


def index_pairs(P, R, L):
    freq = np.zeros(L, np.int64)
    groups = [[] for _ in range(L)]
    for ri, r in enumerate(R):
        for l in items(r):
            freq[l] += 1
            groups[l].append(ri)
    found, tests = set(), 0
    for pi, p in enumerate(P):
        its = items(p)
        key = min(its, key=lambda l: (freq[l], l))
        if freq[key] == 0:
            continue                      # extra group: inside no record
        for ri in groups[key]:
            tests += 1
            if contains(R[ri], p):
                assert (pi, ri) not in found
                found.add((pi, ri))
    return found, tests


@pytest.mark.parametrize("seed", range(8))
def test_index_meets_every_containing_pair_once(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.choice([1, 2, 3]))
    L = 64 * K
    n, m = int(rng.integers(20, 120)), int(rng.integers(20, 120))
    density = float(rng.choice([0.05, 0.15, 0.4]))
    R = [[int(v) for v in row] for row in
         ((rng.random((n, K, 64)) < density) * (1 << np.arange(64, dtype=np.uint64))).sum(
             axis=2, dtype=np.uint64)]
    # Patterns: sub-itemsets of records (many contained somewhere) and random
    # sets (some with an item no record holds).
    P = []
    for _ in range(m):
        if rng.random() < 0.6:
            r = R[int(rng.integers(0, n))]
            p = [w & int(rng.integers(0, 1 << 63)) | 0 for w in r]
        else:
            p = [int(rng.integers(0, 1 << 63)) & int(rng.integers(0, 1 << 63)) for _ in range(K)]
        if any(p):
            P.append(p)
    brute = {(pi, ri) for pi, p in enumerate(P) for ri, r in enumerate(R) if contains(r, p)}
    found, tests = index_pairs(P, R, L)
    assert found == brute
    assert tests <= len(P) * len(R)
    assert brute                                   # the case is not vacuous
