"""Two pieces of the canonical sort (sort.cu), checked on the CPU.

* The order-preserving key prefix: a key's ten highest items, from the top,
  each as (item + 1) in a 12-bit field, five per 64-bit word.  Comparing
  prefixes must never contradict comparing the keys as K-word integers (word
  K-1 most significant): a < b implies prefix(a) <= prefix(b), and
  prefix(a) < prefix(b) implies a < b; equal prefixes are resolved on the
  full keys.  Every prefix word stays below 2^60, under the padding value.
* The block sort's network: a bitonic sort in the flip / disperse form, where
  the first step of stage k pairs position p with p XOR (k - 1) and later
  steps with p XOR j, the lower position keeping the smaller element.  It
  must sort every input, repeated keys included (ties broken by index).
"""
import numpy as np
import pytest


def key_int(words):
    v = 0
    for w in reversed(words):
        v = (v << 64) | int(w)
    return v


def key_prefix(words):
    a = b = 0
    taken = 0
    for w in range(len(words) - 1, -1, -1):
        x = int(words[w])
        while x and taken < 10:
            bit = x.bit_length() - 1
            x &= ~(1 << bit)
            field = w * 64 + bit + 1
            if taken < 5:
                a |= field << (12 * (4 - taken))
            else:
                b |= field << (12 * (9 - taken))
            taken += 1
        if taken >= 10:
            break
    return a, b


def _keys(rng, n, K, density):
    bits = rng.random((n, K, 64)) < density
    words = (bits * (1 << np.arange(64, dtype=np.uint64))).sum(axis=2, dtype=np.uint64)
    return [list(r) for r in words]


@pytest.mark.parametrize("K,density", [(1, 0.05), (2, 0.02), (8, 0.01), (8, 0.2), (16, 0.005)])
def test_prefix_preserves_key_order(K, density):
    rng = np.random.default_rng(K * 1000 + int(density * 1000))
    keys = _keys(rng, 400, K, density)
    # near neighbours too: keys sharing their top items, differing below
    for r in keys[:100]:
        s = list(r)
        s[0] ^= np.uint64(1) << np.uint64(int(rng.integers(0, 64)))
        keys.append(s)
    ints = [key_int(k) for k in keys]
    pre = [key_prefix(k) for k in keys]
    assert all(p < (1 << 60) and q < (1 << 60) for p, q in pre)
    ties = 0
    for i in range(len(keys)):
        for j in range(i + 1, len(keys)):
            if ints[i] < ints[j]:
                assert pre[i] <= pre[j]
            elif ints[j] < ints[i]:
                assert pre[j] <= pre[i]
            if pre[i] < pre[j]:
                assert ints[i] < ints[j]
            elif pre[j] < pre[i]:
                assert ints[j] < ints[i]
            ties += pre[i] == pre[j] and ints[i] != ints[j]
    if density >= 0.2:
        assert ties > 0            # dense keys do share prefixes: the full compare matters


def bitonic_flip_sort(elems):
    C = len(elems)
    el = list(elems)
    k = 2
    while k <= C:
        j = k >> 1
        while j > 0:
            d = k - 1 if j == (k >> 1) else j
            el = [min(el[p], el[p ^ d]) if p < (p ^ d) else max(el[p], el[p ^ d])
                  for p in range(C)]
            j >>= 1
        k <<= 1
    return el


@pytest.mark.parametrize("C", [2, 4, 32, 64, 1024])
def test_block_network_sorts(C):
    rng = np.random.default_rng(C)
    for trial in range(8):
        vals = rng.integers(0, max(2, C // (1 + trial)), C)
        elems = [(int(v), i) for i, v in enumerate(vals)]      # index breaks ties
        assert bitonic_flip_sort(elems) == sorted(elems)
    # a short tile: padding elements (all ones) sort after every real one
    pad = (1 << 64) - 1
    elems = [(int(v), i) for i, v in enumerate(rng.integers(0, 5, C // 2))]
    elems += [(pad, pad)] * (C - len(elems))
    assert bitonic_flip_sort(elems)[:C // 2] == sorted(elems[:C // 2])
