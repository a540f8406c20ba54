"""The canonical sort's merge-pass slot rule, checked on the CPU.

Each merge pass of the sort (sort.cu) merges groups of four sorted runs
without merge-path partitioning: an element of run q goes to slot
  group start + (its index in its run)
             + sum over the group's other runs of the elements before it,
where "before" means smaller, or equal and in a lower run; runs past the end
of the input are empty and the last run may be short.  This test restates
the rule in Python (binary searches bounded as in the kernel) and checks,
with repeated keys and ragged ends, that the slots form a permutation of
[0, n) and that the result is sorted with equal keys in run order.
"""
import bisect

import numpy as np
import pytest

FAN = 4


def merge_pass(v, run):
    n = len(v)
    out = [None] * n
    for e in range(n):
        r = e // run
        own_lo, grp_lo, q = r * run, (r // FAN) * FAN * run, r % FAN
        pos = grp_lo + (e - own_lo)
        for qq in range(FAN):
            if qq == q:
                continue
            a = grp_lo + qq * run
            lo, hi = min(a, n), min(a + run, n)
            seg = v[lo:hi]
            # elements of run qq before v[e]: <= for lower runs, < for higher
            cnt = bisect.bisect_right(seg, v[e]) if qq < q else bisect.bisect_left(seg, v[e])
            pos += cnt
        assert 0 <= pos < n and out[pos] is None, "slot outside the input or taken twice"
        out[pos] = (v[e], e)
    return out


def sort_by_passes(values, tile):
    # Sorted tiles first (as the block sort leaves them), then the passes.
    v = []
    for i in range(0, len(values), tile):
        v += sorted(values[i:i + tile])
    run = tile
    while run < len(v):
        merged = merge_pass(v, run)
        # Each group of FAN runs is now one sorted run, equal keys in the
        # order of their source positions (lower runs first).
        span = FAN * run
        for g in range(0, len(v), span):
            part = merged[g:g + span]
            assert sorted(x for x, _ in part) == sorted(v[g:g + span])
            for (a, ea), (b, eb) in zip(part, part[1:]):
                assert a < b or (a == b and ea < eb)
        v = [x for x, _ in merged]
        run *= FAN
    return v


@pytest.mark.parametrize("n,tile,distinct", [
    (1, 4, 1), (5, 4, 3), (16, 4, 2), (17, 4, 5), (63, 4, 10), (64, 4, 64), (65, 4, 7),
    (300, 8, 20), (1000, 16, 1000), (1023, 16, 3), (4097, 16, 100)])
def test_slots_form_a_sorted_permutation(n, tile, distinct):
    rng = np.random.default_rng(n * 31 + tile)
    values = [int(x) for x in rng.integers(0, distinct, n)]
    assert sort_by_passes(values, tile) == sorted(values)
