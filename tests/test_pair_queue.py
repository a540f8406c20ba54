"""The batched pair stage's device-side tile queue, checked on the CPU.

One launch of the persistent pair kernel (dedup.cu) serves every class of
every problem: the host lays the jobs' tile counts end to end (a job of n
distinct records has nt = ceil(n / 64) tile rows and, from its first band
b0 on, (nt - b0)(nt - b0 + 1) / 2 upper-triangle tiles), and each CTA turns
a queue number q into (job, tile row, tile column) by two binary searches.
This test restates that decoding in Python and checks that every tile
(bi, bj) with b0 <= bi <= bj < nt of every job is met exactly once, and
nothing outside it -- also with empty jobs and jobs that resume at a later
band after their table grew.
"""
import numpy as np
import pytest

TILE = 64


def div_up(a, b):
    return -(-a // b)


def offsets(jobs):
    off = [0]
    for n, b0 in jobs:
        rows = div_up(n, TILE) - b0
        off.append(off[-1] + rows * (rows + 1) // 2)
    return off


def decode(q, jobs, off):
    lo, hi = 0, len(jobs) - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if off[mid] <= q:
            lo = mid
        else:
            hi = mid - 1
    n, b0 = jobs[lo]
    nt = div_up(n, TILE)
    r = q - off[lo]

    def before(b):  # tiles of the bands [b0, b)
        return (b - b0) * nt - (b * (b - 1) // 2 - b0 * (b0 - 1) // 2)

    blo, bhi = b0, nt - 1
    while blo < bhi:
        mid = (blo + bhi + 1) >> 1
        if before(mid) <= r:
            blo = mid
        else:
            bhi = mid - 1
    return lo, blo, blo + (r - before(blo))


def check(jobs):
    off = offsets(jobs)
    got = [decode(q, jobs, off) for q in range(off[-1])]
    want = [(j, bi, bj) for j, (n, b0) in enumerate(jobs)
            for bi in range(b0, div_up(n, TILE)) for bj in range(bi, div_up(n, TILE))]
    assert sorted(got) == want
    return len(got)


@pytest.mark.parametrize("seed", range(10))
def test_random_jobs(seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(int(rng.integers(1, 40))):
        n = int(rng.integers(0, 2000)) if rng.random() > 0.1 else 0
        nt = div_up(n, TILE)
        b0 = int(rng.integers(0, nt)) if nt and rng.random() < 0.3 else 0   # a replayed job
        jobs.append((n, b0))
    check(jobs)


def test_edges():
    assert check([(1, 0)]) == 1                       # one record: one tile
    assert check([(0, 0), (64, 0), (0, 0)]) == 1      # empty jobs around a full tile
    assert check([(65, 0)]) == 3                      # a ragged second tile row
    assert check([(640, 9)]) == 1                     # resumed at the last band
    assert check([(5777, 0), (5166, 0)]) == 91 * 92 // 2 + 81 * 82 // 2   # the 148k classes
