"""Pins for the CPU oracle, against things other than the oracle itself.

* brute force over every itemset of a tiny item universe (tests/brute.py),
* a hand-worked example (tests/golden/hand_worked_L4.json),
* closed forms of special cases (disjoint classes, identical classes, a single
  record, a single one-hot feature, the one-hot encoding of Section 3.1),
* invariants of the definitions on the 500-record workload (subset relations,
  class exclusivity, canonical order, permutation invariance),
* the Regulation 1-3 truth table and the Regulation 3 statistics.

None of these touches the GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import igdata
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ints(rows):
    """uint64[n, K] rows -> Python ints (word K-1 most significant)."""
    out = []
    for r in rows:
        v = 0
        for k in range(len(r) - 1, -1, -1):
            v = (v << 64) | int(r[k])
        out.append(v)
    return out


def _oracle_fit_split(XA, XN):
    rows = np.concatenate([XA, XN])
    lab = np.concatenate([np.ones(len(XA), np.uint8), np.zeros(len(XN), np.uint8)])
    return oracle.fit(rows, lab, threads=2)


def _positions(L, K, start):
    return [start + j for j in range(L)]


def _tiny_case(seed, L, n_attack, n_normal, pool):
    """Itemsets drawn from a small pool so that duplicates occur."""
    rng = np.random.default_rng(seed)
    pool_sets = [int(v) for v in rng.integers(1, 1 << L, size=pool)]
    XA = [pool_sets[i] for i in rng.integers(0, pool, size=n_attack)]
    XN = [pool_sets[i] for i in rng.integers(0, pool, size=n_normal)]
    return XA, XN


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("layout", ["one_word", "straddle"])
def test_brute_force_fit_and_score(seed, layout):
    L = 10 if seed % 2 else 12
    if layout == "one_word":
        K, positions = 1, _positions(L, 1, 0)
    else:  # items at bit positions 58..69: across the word-0/word-1 boundary
        K, positions = 2, _positions(L, 2, 58)
    XA, XN = _tiny_case(seed, L, 3 + seed % 8, 2 + (seed * 7) % 9,
                        pool=6 + seed % 5)
    want = brute.fit(XA, XN, L)
    model = _oracle_fit_split(brute.pack(XA, positions, K),
                              brute.pack(XN, positions, K))
    for cls in (1, 0):
        B, P, f, S = want[cls]
        X = XA if cls == 1 else XN
        got_B = oracle.candidates(brute.pack(X, positions, K))
        assert got_B.shape[0] == len(B) == model.n_candidates[cls]
        np.testing.assert_array_equal(got_B, brute.pack(B, positions, K))
        np.testing.assert_array_equal(model.patterns[cls],
                                      brute.pack(P, positions, K).reshape(-1, K))
        np.testing.assert_array_equal(model.support[cls], np.asarray(f, np.uint32))
        np.testing.assert_array_equal(model.score[cls], np.asarray(S, np.uint64))
    # Eq. 4 and Regulations 1-2 on every itemset of the universe.
    tests = list(range(0, 1 << L, 7))
    A, N, lab = oracle.score(model, brute.pack(tests, positions, K))
    for i, t in enumerate(tests):
        a = brute.evidence(want[1][1], want[1][3], t)
        n = brute.evidence(want[0][1], want[0][3], t)
        assert (A[i], N[i], lab[i]) == (a, n, brute.label(a, n))


def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "hand_worked_L4.json")))
    letter = {"a": 1, "b": 2, "c": 4, "d": 8}

    def rows(names):
        return np.array([[sum(letter[ch] for ch in s)] for s in names], np.uint64)

    XA, XN = rows(g["attack_records"]), rows(g["normal_records"])
    m = _oracle_fit_split(XA, XN)
    assert m.n_candidates[1] == g["n_candidates_attack"]
    assert m.n_candidates[0] == g["n_candidates_normal"]
    assert m.patterns[1][:, 0].tolist() == g["P_attack"]
    assert m.support[1].tolist() == g["f_attack"]
    assert m.score[1].tolist() == g["S_attack"]
    assert m.patterns[0][:, 0].tolist() == g["P_normal"]
    assert m.support[0].tolist() == g["f_normal"]
    assert m.score[0].tolist() == g["S_normal"]
    A, N, lab = oracle.score(m, rows(g["test_records"]))
    assert A.tolist() == g["A"] and N.tolist() == g["N"]
    assert lab.tolist() == g["labels"]
    all_rows = np.concatenate([XA, XN])
    all_lab = np.array([1] * len(XA) + [0] * len(XN), np.uint8)
    m3 = oracle.fit(all_rows, all_lab, r=g["reg3_r"])
    mu, sigma, r, thr = m3.reg3
    assert (mu, sigma, thr) == (g["reg3_mu"], g["reg3_sigma"], g["reg3_threshold"])
    assert oracle.score(m3, rows(g["test_records"]))[2].tolist() == g["labels_reg3"]


def test_encode_closed_form():
    # Section 3.1: item of (feature f, value v) = sum of earlier cards + v.
    cards = np.array([3, 70, 11], np.uint16)
    codes = np.array([[2, 0, 10], [0, 69, 0], [1, 5, 3]], np.uint16)
    rows = oracle.encode(codes, cards)
    assert rows.shape == (3, 2)                      # L = 84 -> K = 2
    assert _ints(rows) == [(1 << 2) | (1 << 3) | (1 << 83),
                           (1 << 0) | (1 << 72) | (1 << 73),
                           (1 << 1) | (1 << 8) | (1 << 76)]
    with pytest.raises(ValueError):
        oracle.encode(np.array([[3, 0, 0]], np.uint16), cards)


def test_encode_missing_value_has_no_item():
    cards = np.array([3, 70, 11], np.uint16)
    codes = np.array([[2, 0xFFFF, 10], [0xFFFF, 0xFFFF, 0xFFFF]], np.uint16)
    assert _ints(oracle.encode(codes, cards)) == [(1 << 2) | (1 << 83), 0]


def test_encode_one_hot_properties():
    w = igdata.nsl15k()
    rows = oracle.encode(w.train_codes[:500], w.cards)
    assert rows.shape[1] == 8
    offsets = np.concatenate([[0], np.cumsum(w.cards.astype(np.int64))])
    for r, codes in zip(_ints(rows), w.train_codes[:500]):
        assert bin(r).count("1") == w.n_features
        assert r >> w.n_items == 0                    # tail bits stay zero
        for f in range(w.n_features):
            field = (r >> int(offsets[f])) & ((1 << int(w.cards[f])) - 1)
            assert field == 1 << int(codes[f])


def test_disjoint_classes_every_candidate_coherent():
    # Attack records use items 0..5, normal records items 6..11: nothing of
    # one class can lie inside a record of the other.
    rng = np.random.default_rng(5)
    XA = [int(v) for v in rng.integers(1, 64, size=9)]
    XN = [int(v) << 6 for v in rng.integers(1, 64, size=8)]
    m = _oracle_fit_split(brute.pack(XA, range(12), 1), brute.pack(XN, range(12), 1))
    for cls, X in ((1, XA), (0, XN)):
        expected = {x for x in X} | {X[i] & X[j] for i in range(len(X))
                                     for j in range(i + 1, len(X))}
        expected.discard(0)
        assert m.n_candidates[cls] == len(expected)
        assert sorted(expected) == _ints(m.patterns[cls])


def test_identical_classes_nothing_coherent():
    rng = np.random.default_rng(6)
    X = brute.pack([int(v) for v in rng.integers(1, 1 << 10, size=7)], range(10), 1)
    m = _oracle_fit_split(X, X[::-1].copy())
    assert m.patterns[1].shape[0] == 0 and m.patterns[0].shape[0] == 0
    A, N, lab = oracle.score(m, X)
    assert (A == 0).all() and (N == 0).all() and (lab == 1).all()   # Regulation 2


def test_single_record_class():
    x = np.array([[0b1011]], np.uint64)
    assert _ints(oracle.candidates(x)) == [0b1011]
    assert oracle.candidates(np.zeros((1, 1), np.uint64)).shape[0] == 0


def test_single_one_hot_feature():
    # One feature: two distinct values never share an item, so B^c is the set
    # of distinct records, and P^c those values absent from the other class;
    # f counts the copies of the value in its own class.
    rng = np.random.default_rng(7)
    cards = np.array([12], np.uint16)
    ca = rng.integers(0, 12, size=(30, 1)).astype(np.uint16)
    cn = rng.integers(0, 12, size=(25, 1)).astype(np.uint16)
    m = _oracle_fit_split(oracle.encode(ca, cards), oracle.encode(cn, cards))
    for cls, own, other in ((1, ca, cn), (0, cn, ca)):
        vals = sorted(set(own[:, 0].tolist()) - set(other[:, 0].tolist()))
        assert _ints(m.patterns[cls]) == [1 << v for v in vals]
        assert m.support[cls].tolist() == [int((own[:, 0] == v).sum()) for v in vals]
        assert m.score[cls].tolist() == m.support[cls].tolist()      # |b| = 1


@pytest.fixture(scope="module")
def tiny_fit():
    w = igdata.tiny()
    rows = oracle.encode(w.train_codes, w.cards)
    return w, rows, oracle.fit(rows, w.train_labels)


def test_invariants_tiny(tiny_fit):
    w, rows, m = tiny_fit
    X = {c: _ints(rows[w.train_labels == c]) for c in (0, 1)}
    for cls in (1, 0):
        P = _ints(m.patterns[cls])
        assert P == sorted(set(P))                                # canonical, unique
        for b, f in zip(P, m.support[cls]):
            holders = [x for x in X[cls] if brute.contains(x, b)]
            assert len(holders) == f >= 1                          # Eq. 2 support
            if b not in X[cls]:                                    # a pair intersection
                assert f >= 2
            assert not any(brute.contains(y, b) for y in X[1 - cls])   # Eq. 3
            assert bin(b).count("1") <= w.n_features
    assert not set(_ints(m.patterns[0])) & set(_ints(m.patterns[1]))
    # Every nonempty pairwise intersection of the same class is a candidate:
    # it is kept exactly when no opposite record contains it.
    rng = np.random.default_rng(8)
    for cls in (1, 0):
        Xc, P = X[cls], set(_ints(m.patterns[cls]))
        for _ in range(300):
            i, j = rng.integers(0, len(Xc), size=2)
            b = Xc[i] & Xc[j]
            coh = b != 0 and not any(brute.contains(y, b) for y in X[1 - cls])
            assert (b in P) == coh


def test_permutation_invariance(tiny_fit):
    w, rows, m = tiny_fit
    perm = np.random.default_rng(9).permutation(rows.shape[0])
    m2 = oracle.fit(rows[perm], w.train_labels[perm])
    for cls in (0, 1):
        np.testing.assert_array_equal(m.patterns[cls], m2.patterns[cls])
        np.testing.assert_array_equal(m.support[cls], m2.support[cls])
        np.testing.assert_array_equal(m.score[cls], m2.score[cls])


def test_training_attack_record_evidence(tiny_fit):
    # A training attack record x that is itself coherent contributes S+(x) to
    # its own A(x), so A(x) >= S+(x).
    w, rows, m = tiny_fit
    P = {b: s for b, s in zip(_ints(m.patterns[1]), m.score[1].tolist())}
    XA = rows[w.train_labels == 1]
    A, _, _ = oracle.score(m, XA)
    hits = 0
    for x, a in zip(_ints(XA), A):
        if x in P:
            hits += 1
            assert a >= P[x]
    assert hits > 0


def test_labels_truth_table():
    A = np.array([0, 1, 0, 5, 3, 3, 2, 9])
    N = np.array([0, 0, 1, 5, 7, 7, 1, 20])
    # R2, R1, R1, R1 tie, R3 fires (7 < 10), R3 silent (7 >= 5), R1, R3 fires
    assert oracle.labels(A, N).tolist() == [1, 1, 0, 1, 0, 0, 1, 0]
    np.testing.assert_array_equal(oracle.labels(A[:5], N[:5], 10.0), [1, 1, 1, 1, 1])
    np.testing.assert_array_equal(oracle.labels(A[4:6], N[4:6], 5.0), [0, 0])
    np.testing.assert_array_equal(oracle.labels(A[7:], N[7:], 20.5), [1])
    np.testing.assert_array_equal(oracle.labels(A[7:], N[7:], 20.0), [0])   # strict <


def test_reg3_statistics_closed_form():
    mu, sigma = oracle.reg3_stats(np.array([1, 2, 3, 4]))
    assert mu == 2.5 and sigma == math.sqrt(1.25)                # population std
    mu, sigma = oracle.reg3_stats(np.array([5, 5, 5]))
    assert (mu, sigma) == (5.0, 0.0)
    assert oracle.reg3_threshold(2.5, 0.5, 3.0) == 1.0


def test_pattern_score_for_given_supports():
    # Eq. 2 with the supports given: |b| counts items in every word (an item
    # in word 0 and one in the top bit of word 1 make |b| = 2).
    P = np.array([[0b10110, 0], [1, 1 << 63], [0, 0b111]], np.uint64)
    f = np.array([5, 2, 7], np.uint32)
    assert oracle.pattern_score(P, f).tolist() == [5 * 9, 2 * 4, 7 * 9]
    # The same scores as the support step's own (brute-force pinned) ones.
    rng = np.random.default_rng(21)
    same = igdata.random_words(rng, 60, 150, "half")
    pats = same[rng.integers(0, 60, size=25)] & same[rng.integers(0, 60, size=25)]
    pats = pats[np.any(pats != 0, axis=1)]
    fs, S = oracle.support(pats, same)
    assert np.array_equal(oracle.pattern_score(pats, fs), S)


def test_model_from_patterns_canonical_order():
    # Given dictionaries come back ascending as K-word integers (word K-1
    # most significant), supports following their patterns.
    P = np.array([[5, 1], [7, 0], [1, 1], [2, 0]], np.uint64)
    m = oracle.model_from_patterns({0: P, 1: P[:2]}, {0: [10, 20, 30, 40], 1: [1, 2]})
    assert m.patterns[0].tolist() == [[2, 0], [7, 0], [1, 1], [5, 1]]
    assert m.support[0].tolist() == [40, 20, 30, 10]
    assert m.score[0].tolist() == [40 * 1, 20 * 9, 30 * 4, 10 * 9]
    assert m.patterns[1].tolist() == [[7, 0], [5, 1]]


def test_evidence_sums_beyond_32_bits():
    # Eq. 4 closed form: a record holding every item of one word contains
    # every pattern made of its items, so its evidence is the sum of all the
    # patterns' scores.  2,081 patterns of 62-64 items with support 1,000
    # score 3.8-4.1 million each: the sum is about 8e9, beyond 32 bits.
    from itertools import combinations
    full = (1 << 64) - 1
    pats = [full] + [full ^ (1 << a) for a in range(64)] + \
           [full ^ (1 << a) ^ (1 << b) for a, b in combinations(range(64), 2)]
    P = np.array([[p] for p in pats], np.uint64)
    f = np.full(len(pats), 1000, np.uint32)
    S = oracle.pattern_score(P, f)
    want = sum(1000 * bin(p).count("1") ** 2 for p in pats)
    assert want > 2 ** 32 and int(S.astype(object).sum()) == want
    got = oracle.evidence(P, S, np.array([[full], [full ^ 1]], np.uint64))
    assert got.dtype == np.int64
    # the second record lacks item 0: only patterns without it are inside
    assert got.tolist() == [want, sum(1000 * bin(p).count("1") ** 2 for p in pats if not p & 1)]


def test_score_applies_regulation3(tiny_fit):
    # Scoring with a fitted Regulation 3: labels follow Regulations 1-3 with
    # the model's threshold, applied here by hand to the oracle's (brute-force
    # pinned) evidence, and some normal-by-Regulation-1 records do turn attack.
    w, rows, _ = tiny_fit
    m = oracle.fit(rows, w.train_labels, r=0.5)
    test = oracle.encode(w.test_codes, w.cards)
    A, N, lab = oracle.score(m, test)
    assert np.array_equal(A, oracle.evidence(m.patterns[1], m.score[1], test))
    assert np.array_equal(N, oracle.evidence(m.patterns[0], m.score[0], test))
    thr = m.reg3[3]
    want = [1 if (a >= n or (a == 0 and n == 0) or float(n) < thr) else 0
            for a, n in zip(A.tolist(), N.tolist())]
    assert lab.tolist() == want
    assert sum(1 for a, n in zip(A.tolist(), N.tolist()) if a < n and float(n) < thr) > 0
