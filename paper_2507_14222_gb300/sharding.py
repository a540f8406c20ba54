"""Host-side bookkeeping of the sharded (multi-GPU) form of IG training.

Not run on GPUs here: every call of this build sees one GPU, so the sharded
path is a design, and this module holds the parts of it that decide who
does what, tested with gloo ranks on the CPU.  The design, per class c with
records X^c replicated on every rank (they are small: 7,844 x 64 B at the
148k shape):

1. Pairs (Eq. 1).  The upper triangle of pair tiles is cut into W bands of
   whole tile rows holding about equal numbers of pairs (pair_bands); rank r
   intersects the pairs of band r and deduplicates them in its own table.
2. Owners.  Every rank draws a sample of its distinct keys; the samples are
   gathered and W - 1 splitters picked from them in canonical order
   (ascending as K-word integers, word K-1 most significant; splitters).
   Key b belongs to the rank whose splitter range holds it (owner_of), so
   the owners hold contiguous ranges of the canonical order.
3. Exchange.  A distinct key travels to its owner as its pair (i, j) -- 8
   bytes, as the records are replicated -- in one all-to-all; the owner
   recomputes x_i AND x_j and deduplicates again (a key made on two ranks
   arrives twice).
4. Coherence and supports (Eq. 3, Eq. 2).  Each owner tests its shard
   against the replicated records of both classes: no communication.
5. Canonical order.  Each owner sorts its shard; the single-GPU canonical
   list is the concatenation of the shards in rank order (merge_shards), as
   the ranges do not overlap.
6. Evidence (Eq. 4).  Each owner scores all test records against its shard
   of P^c; the int64 partial sums A and N (m x 8 bytes each) are summed by
   one all-reduce (integer sums: the order of addition does not matter).
   Regulation 3's mu_N and sigma_N come from the all-reduced N of the
   training normals, computed on every rank in record order as on one GPU.

Message sizes per step are estimated by exchange_bytes.
"""
from __future__ import annotations

import bisect

import numpy as np

PAIR_TILE = 64  # records per side of a pair tile (one band row = one tile row)


def key_int(row) -> int:
    """A K-word key as one integer, word K-1 most significant (the
    canonical order of pattern lists)."""
    v = 0
    for w in reversed([int(x) for x in row]):
        v = (v << 64) | w
    return v


def pair_bands(n: int, world: int, tile: int = PAIR_TILE) -> list:
    """Cuts the tile rows of the upper triangle of an n x n pair matrix
    (pairs i <= j, the diagonal giving the records themselves) into `world`
    bands [lo, hi) of whole tile rows with about equal numbers of pairs.
    Tile row t pairs records [t*tile, (t+1)*tile) with records >= t*tile."""
    nt = (n + tile - 1) // tile
    # pairs of tile row t: its rows against every record from its first on
    weight = []
    for t in range(nt):
        lo, hi = t * tile, min(n, (t + 1) * tile)
        weight.append(sum(n - i for i in range(lo, hi)))
    total = sum(weight)
    cum = [0]
    for wt in weight:
        cum.append(cum[-1] + wt)
    # Cut r (r = 1 .. W-1) at the tile-row boundary whose cumulative pair
    # count is nearest to r/W of the total.
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        t = bisect.bisect_left(cum, target)
        if t > 0 and (t > nt or abs(cum[t - 1] - target) <= abs(cum[t] - target)):
            t -= 1
        cuts.append(max(cuts[-1], min(t, nt)))
    cuts.append(nt)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def band_pairs(n: int, band: tuple, tile: int = PAIR_TILE):
    """The pairs (i, j), i <= j, of the tile rows [band[0], band[1])."""
    for t in range(band[0], band[1]):
        for i in range(t * tile, min(n, (t + 1) * tile)):
            for j in range(i, n):
                yield i, j


def splitters(samples: list, world: int) -> list:
    """W - 1 splitters (key integers) from the gathered samples: the keys at
    the quantiles 1/W, 2/W, ... of the sorted sample."""
    s = sorted(set(samples))
    if not s:
        return [0] * (world - 1)
    return [s[min(len(s) - 1, (len(s) * r) // world)] for r in range(1, world)]


def owner_of(key: int, split: list) -> int:
    """The rank whose range [split[r-1], split[r]) holds the key."""
    return bisect.bisect_right(split, key)


def merge_shards(shards: list) -> list:
    """The canonical list from the owners' sorted shards: their
    concatenation in rank order (checked to be ascending)."""
    out = [k for sh in shards for k in sh]
    if any(out[i] >= out[i + 1] for i in range(len(out) - 1)):
        raise ValueError("shards overlap or are not sorted")
    return out


def exchange_bytes(local_distinct: list, m_test: int) -> dict:
    """Bytes moved per class and fit + score: the pair ids of every rank's
    distinct keys (8 bytes each) in the all-to-all, and the all-reduce of the
    int64 evidence sums A and N over m_test records."""
    return {"all_to_all": 8 * int(sum(local_distinct)), "all_reduce": 2 * 8 * int(m_test)}
