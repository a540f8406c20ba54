"""Bookkeeping of the sharded form of IG training (design only: no call of
this build sees more than one GPU), run as two gloo ranks on the CPU.

Each rank intersects the pairs of its band (Eq. 1), deduplicates them,
draws a sample, and the gathered samples give the splitters; every distinct
key goes to its owner as its pair (i, j) in one all-to-all, the owner
recomputes and deduplicates it, and the owners' sorted shards, concatenated
in rank order, must equal the single-process candidate list of the CPU
oracle -- every candidate on exactly one owner, in canonical order.  The
evidence step's all-reduce of partial sums must give the oracle's A.  A
second test runs the whole sharded fit and score of a two-class problem --
owners' coherence and support steps on the replicated records, the
all-reduced A and N, Regulation 3's statistics -- against the single-process
oracle fit.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import igdata
import oracle
from paper_2507_14222_gb300 import sharding


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _records():
    rng = np.random.default_rng(31)
    base = igdata.random_words(rng, 90, 130, "quarter")
    return base[rng.integers(0, 90, size=150)]          # duplicates occur


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X = _records()
        n = X.shape[0]
        band = sharding.pair_bands(n, world, tile=16)[rank]
        local = {}
        for i, j in sharding.band_pairs(n, band, tile=16):
            b = X[i] & X[j]
            if b.any():
                local.setdefault(sharding.key_int(b), (i, j))
        keys = sorted(local)
        sample = keys[::7]
        gathered = [None] * world
        dist.all_gather_object(gathered, sample)
        split = sharding.splitters([k for s in gathered for k in s], world)
        # All-to-all of pair ids, routed by owner.
        outbox = [[] for _ in range(world)]
        for k in keys:
            outbox[sharding.owner_of(k, split)].append(local[k])
        inbox = [None] * world
        for dst in range(world):
            got = [None] * world
            dist.all_gather_object(got, outbox[dst])
            if dst == rank:
                inbox = got
        shard = set()
        for src in range(world):
            for i, j in inbox[src]:
                k = sharding.key_int(X[i] & X[j])
                assert sharding.owner_of(k, split) == rank
                shard.add(k)
        shard = sorted(shard)
        # Evidence: this owner's partial A over all records, all-reduced.
        pats = [k for k in shard]
        P = np.array([[(k >> (64 * w)) & ((1 << 64) - 1) for w in range(X.shape[1])]
                      for k in pats], dtype=np.uint64).reshape(-1, X.shape[1])
        S = np.arange(1, P.shape[0] + 1, dtype=np.uint64) * np.uint64(rank + 1)
        part = torch.from_numpy(oracle.evidence(P, S, X))
        dist.all_reduce(part)
        out[rank] = (shard, len(keys), [int(v) for v in part.tolist()],
                     [int(k) for k in pats], [int(v) for v in S.tolist()])
    finally:
        dist.destroy_process_group()


def test_sharded_candidates_merge_to_single_process_order():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    X = _records()
    want = [sharding.key_int(r) for r in oracle.candidates(X)]
    shards = [res[r][0] for r in range(world)]
    assert all(len(s) for s in shards)                       # both ranks own keys
    merged = sharding.merge_shards(shards)
    assert merged == want                                     # one owner each, canonical
    # Every rank holds the same all-reduced evidence: the sum over both
    # owners' patterns, as one process would compute it.
    pats = res[0][3] + res[1][3]
    S = res[0][4] + res[1][4]
    K = X.shape[1]
    P = np.array([[(k >> (64 * w)) & ((1 << 64) - 1) for w in range(K)] for k in pats],
                 dtype=np.uint64)
    A = oracle.evidence(P, np.array(S, np.uint64), X)
    assert res[0][2] == res[1][2] == A.tolist()
    sizes = sharding.exchange_bytes([res[r][1] for r in range(world)], X.shape[0])
    assert sizes["all_to_all"] == 8 * (res[0][1] + res[1][1])


def _labelled():
    """Records of two classes (K = 3, duplicates within and across classes)
    and separate test records."""
    rng = np.random.default_rng(37)
    base = igdata.random_words(rng, 100, 130, "quarter")
    X = base[rng.integers(0, 100, size=170)]
    y = (rng.random(170) < 0.45).astype(np.uint8)
    T = base[rng.integers(0, 100, size=60)] | igdata.random_words(rng, 60, 130, "quarter")
    return X, y, T


def _words(keys, K):
    return np.array([[(k >> (64 * w)) & ((1 << 64) - 1) for w in range(K)] for k in keys],
                    dtype=np.uint64).reshape(-1, K)


def _exchange(outbox, rank, world):
    """All-to-all of Python lists, as one all_gather per destination."""
    inbox = None
    for dst in range(world):
        got = [None] * world
        dist.all_gather_object(got, outbox[dst])
        if dst == rank:
            inbox = got
    return inbox


def _rank_fit(rank, world, port, r, out):
    # Every step of the sharded fit and score, one class at a time.
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, y, T = _labelled()
        K = X.shape[1]
        Xc = {c: X[y == c] for c in (0, 1)}
        mine = {}
        for c in (0, 1):
            R = Xc[c]
            # 1. this rank's band of pairs, deduplicated locally
            local = {}
            for i, j in sharding.band_pairs(R.shape[0],
                                            sharding.pair_bands(R.shape[0], world, tile=16)[rank],
                                            tile=16):
                b = R[i] & R[j]
                if b.any():
                    local.setdefault(sharding.key_int(b), (i, j))
            keys = sorted(local)
            # 2. owners from the gathered samples
            gathered = [None] * world
            dist.all_gather_object(gathered, keys[::5])
            split = sharding.splitters([k for g in gathered for k in g], world)
            # 3. each distinct key to its owner as its pair
            outbox = [[] for _ in range(world)]
            for k in keys:
                outbox[sharding.owner_of(k, split)].append(local[k])
            shard = sorted({sharding.key_int(R[i] & R[j])
                            for src in _exchange(outbox, rank, world) for i, j in src})
            # 4. coherence against the other class, supports in this class:
            # the owner alone, on the replicated records
            B = _words(shard, K)
            P = np.ascontiguousarray(B[oracle.coherent(B, Xc[1 - c])])
            f, S = oracle.support(P, Xc[c])
            mine[c] = (P, f, S, len(shard))
        # 6. evidence: this owner's partial sums, all-reduced; Regulation 3
        # statistics from the all-reduced N of the training normals
        parts = [torch.from_numpy(oracle.evidence(mine[1][0], mine[1][2], T)),
                 torch.from_numpy(oracle.evidence(mine[0][0], mine[0][2], T)),
                 torch.from_numpy(oracle.evidence(mine[0][0], mine[0][2], Xc[0]))]
        for t in parts:
            dist.all_reduce(t)
        A, N, n_train = (t.numpy() for t in parts)
        mu, sigma = oracle.reg3_stats(n_train)
        thr = oracle.reg3_threshold(mu, sigma, r)
        out[rank] = ({c: ([sharding.key_int(b) for b in mine[c][0]], mine[c][1].tolist(),
                          mine[c][2].tolist(), mine[c][3]) for c in (0, 1)},
                     A.tolist(), N.tolist(), oracle.labels(A, N, thr).tolist(), (mu, sigma, thr))
    finally:
        dist.destroy_process_group()


def test_sharded_fit_equals_single_process_fit():
    world, r = 2, 0.5
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_fit, args=(world, port, r, out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    X, y, T = _labelled()
    m = oracle.fit(X, y, r=r)
    for c in (0, 1):
        per = [res[k][0][c] for k in range(world)]
        assert all(len(p[0]) for p in per)                       # both owners keep patterns
        # 5. canonical order: the owners' shards in rank order
        assert sharding.merge_shards([p[0] for p in per]) == \
            [sharding.key_int(b) for b in m.patterns[c]]
        assert [v for p in per for v in p[1]] == m.support[c].tolist()
        assert [v for p in per for v in p[2]] == m.score[c].tolist()
        assert sum(p[3] for p in per) == m.n_candidates[c]      # every candidate owned once
    A, N, lab = oracle.score(m, T)
    for k in range(world):                                      # the same on every rank
        assert res[k][1] == A.tolist() and res[k][2] == N.tolist()
        assert res[k][3] == lab.tolist()
        assert res[k][4] == (m.reg3[0], m.reg3[1], m.reg3[3])


def test_pair_bands_cover_every_pair_once():
    for n, world in ((1, 2), (17, 2), (150, 3), (300, 8)):
        bands = sharding.pair_bands(n, world, tile=16)
        assert len(bands) == world and bands[0][0] == 0
        assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
        got = [p for b in bands for p in sharding.band_pairs(n, b, tile=16)]
        assert sorted(got) == [(i, j) for i in range(n) for j in range(i, n)]
    # Balanced by pairs to within about half a tile row's pairs.
    counts = [sum(1 for _ in sharding.band_pairs(4000, b)) for b in sharding.pair_bands(4000, 4)]
    assert max(counts) - min(counts) <= 64 * 4000


def test_owner_ranges_follow_canonical_order():
    keys = list(range(0, 1000, 3))
    split = sharding.splitters(keys, 4)
    owners = [sharding.owner_of(k, split) for k in keys]
    assert owners == sorted(owners) and set(owners) == {0, 1, 2, 3}
    row = np.array([5, 1], np.uint64)                         # word 1 most significant
    assert sharding.key_int(row) == (1 << 64) | 5
    with pytest.raises(ValueError):
        sharding.merge_shards([[1, 5], [3]])
