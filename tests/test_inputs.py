"""The seeded synthetic workloads have the shapes the input recipe states.

Sizes, splits, feature cardinalities and code ranges of every workload, the
batched problems' ranges, the served workload's structure (on a small
instance), and determinism: a workload is a pure function of its seed.  CPU
only; none of the method's arithmetic is involved.
"""
import numpy as np
import pytest

import igdata

MISSING = 0xFFFF


def _check_codes(codes, cards):
    assert codes.dtype == np.uint16 and codes.shape[1] == cards.shape[0]
    assert (codes < cards[None, :]).all()


@pytest.mark.parametrize("make,n_normal,n_attack,n_test,cards,K", [
    (igdata.tiny, 250, 250, 2000, [16] * 16, 4),
    (igdata.nsl15k, 3975, 3525, 7500, igdata.NSL_CARDS, 8),
    (igdata.nsl148k, 7844, 6956, 133200, igdata.NSL_CARDS, 8),
], ids=["tiny", "nsl15k", "nsl148k"])
def test_workload_shapes(make, n_normal, n_attack, n_test, cards, K):
    w = make()
    assert w.cards.tolist() == list(cards)
    assert w.n_items == sum(cards) and w.n_words == K
    assert np.bincount(w.train_labels, minlength=2).tolist() == [n_normal, n_attack]
    assert w.test_codes.shape[0] == n_test == w.test_labels.shape[0]
    assert int((w.test_labels == 0).sum()) == round(0.53 * n_test)         # 53% normal
    _check_codes(w.train_codes, w.cards)
    _check_codes(w.test_codes, w.cards)
    again = make()
    assert np.array_equal(again.train_codes, w.train_codes)
    assert np.array_equal(again.test_codes, w.test_codes)
    assert np.array_equal(again.train_labels, w.train_labels)


def test_nsl_splits():
    # 15k: 50/50 train/test; 148k: 10/90, both 53% normal overall.
    w15, w148 = igdata.nsl15k(), igdata.nsl148k()
    assert w15.train_codes.shape[0] == w15.test_codes.shape[0] == 7500
    n148 = w148.train_codes.shape[0] + w148.test_codes.shape[0]
    assert n148 == 148000 and w148.train_codes.shape[0] == 14800
    normal = int((w148.train_labels == 0).sum() + (w148.test_labels == 0).sum())
    assert abs(normal / n148 - 0.53) < 1e-3


def test_batched_problems():
    widths, sizes = set(), []
    for i in range(igdata.BATCHED_PROBLEMS):
        w = igdata.batched_problem(i)
        n = w.train_codes.shape[0] + w.test_codes.shape[0]
        sizes.append(n)
        assert 200 <= n <= 8000
        assert w.n_items in (128, 256, 512, 1024) and w.cards.tolist() == [16] * (w.n_items // 16)
        widths.add(w.n_items)
        frac = float(np.concatenate([w.train_labels, w.test_labels]).mean())
        assert 0.25 <= frac <= 0.75                      # U[0.3, 0.7] plus sampling noise
        assert set(np.unique(w.train_labels).tolist()) == {0, 1}
        assert abs(w.test_codes.shape[0] - 0.1 * n) <= 1
        _check_codes(w.train_codes, w.cards)
        _check_codes(w.test_codes, w.cards)
    assert widths == {128, 256, 512, 1024}
    assert min(sizes) < 600 and max(sizes) > 5000             # log-uniform spread
    assert len({igdata.batched_problem(i).name for i in range(igdata.BATCHED_PROBLEMS)}) == 64


def test_served_structure_small():
    sw = igdata.served(per_class=3000, total_flows=20000, seed=77)
    for c in (0, 1):
        P = sw.patterns[c]
        assert P.shape == (3000, len(igdata.NSL_CARDS))
        assert np.unique(P, axis=0).shape[0] == 3000       # distinct as code rows
        present = P != MISSING
        assert present.any(axis=1).all()                   # at least one feature kept
        assert (P[present] < np.broadcast_to(sw.cards, P.shape)[present]).all()
        f = sw.support[c]
        assert f.dtype == np.uint32 and f.min() >= 1 and f.max() <= 1000
    assert sw.flow_codes.shape == (20000, len(igdata.NSL_CARDS))
    _check_codes(sw.flow_codes, sw.cards)
    assert int(sw.request_sizes.sum()) == 20000
    assert sw.request_sizes.min() >= 1 and sw.request_sizes.max() <= 4096
    assert sw.unit_gaps.shape == sw.request_sizes.shape and (sw.unit_gaps > 0).all()
    again = igdata.served(per_class=3000, total_flows=20000, seed=77)
    assert all(np.array_equal(again.patterns[c], sw.patterns[c]) for c in (0, 1))
    assert np.array_equal(again.request_sizes, sw.request_sizes)
