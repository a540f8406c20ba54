"""Pins of the oracle's host helpers (preprocessing and evaluation) to values
fixed by hand, closed forms, brute force and a library routine -- never to
the CUDA library.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import helpers as H

NAN = float("nan")


# ---- discretiser (Section 3.1: z-score, round to p decimals, tokens) --------

def test_population_statistics_closed_form():
    # [0, 2]: mean 1, population deviation 1 (the sample one would be sqrt 2).
    assert H._column_stats(np.array([0.0, 2.0])) == (1.0, 1.0)
    # [-2, 2, -1, 1, -1, 1, 0 x 6]: mean 0, sum of squares 12 over 12 -> 1.
    col = np.array([-2, 2, -1, 1, -1, 1, 0, 0, 0, 0, 0, 0], float)
    assert H._column_stats(col) == (0.0, 1.0)
    # Missing entries are left out of both sums.
    assert H._column_stats(np.array([NAN, 0.0, np.inf, 2.0])) == (1.0, 1.0)


def test_token_rounds_half_to_even():
    # mu 0, sigma 1, p = 1: z * 10 = 2.5 -> 2, 7.5 -> 8, -2.5 -> -2, 1.25 * 10 = 12.5 -> 12
    tok = [H._token(x, False, 0.0, 1.0, 10.0) for x in (0.25, 0.75, -0.25, 1.25, 0.3)]
    assert tok == [2, 8, -2, 12, 3]
    # sigma 2, mu 1: z = (4 - 1) / 2 = 1.5 -> p = 0 gives 2
    assert H._token(4.0, False, 1.0, 2.0, 1.0) == 2
    assert H._token(NAN, False, 0.0, 1.0, 1.0) is None
    assert H._token(5.0, False, 5.0, 0.0, 1.0) == 0      # zero deviation
    assert H._token(-0.0, True, 0, 0, 1) == 0.0            # categorical: as is
    assert H._token(7.0, True, 0, 0, 1) == 7.0


def test_discretize_hand_example():
    # Column 0 numeric [1, 2, 3, 4]: mean 2.5, sd sqrt(1.25) = 1.118;
    # z = -1.342, -0.447, 0.447, 1.342 -> p = 0 tokens -1, 0, 0, 1 -> codes 0 1 1 2.
    # Column 1 categorical [7, 3, 7, 9] -> vocabulary 3 < 7 < 9 -> codes 1 0 1 2.
    fit = np.array([[1, 7], [2, 3], [3, 7], [4, 9]], float)
    codes, cards = H.discretize(fit, [False, True], 0)
    assert codes.tolist() == [[0, 1], [1, 0], [1, 1], [2, 2]]
    assert cards.tolist() == [3, 3]
    # p = 1: tokens -13, -4, 4, 13 -> four codes.
    codes, cards = H.discretize(fit, [False, True], 1)
    assert codes[:, 0].tolist() == [0, 1, 2, 3] and cards[0] == 4
    # Coding other rows: a token the fit rows never had, or NaN, is missing.
    vals = np.array([[2.6, 9], [100.0, 5], [NAN, NAN]])
    codes, _ = H.discretize(fit, [False, True], 0, values=vals)
    assert codes.tolist() == [[1, 2], [0xFFFF, 0xFFFF], [0xFFFF, 0xFFFF]]


def test_discretize_invariances():
    rng = np.random.default_rng(5)
    x = rng.integers(-20, 20, size=(64, 3)).astype(float)   # exact sums (n = 64)
    base, cards = H.discretize(x, [False] * 3, 1)
    # A shift by an integer leaves every deviation exact: same codes.
    assert np.array_equal(H.discretize(x + 7.0, [False] * 3, 1)[0], base)
    # Scaling by a power of two scales mean and deviation exactly: same codes.
    assert np.array_equal(H.discretize(x * 4.0, [False] * 3, 1)[0], base)
    # Negation negates every token (half-to-even is symmetric): ranks reverse.
    neg, cards_n = H.discretize(-x, [False] * 3, 1)
    assert np.array_equal(cards_n, cards)
    assert np.array_equal(neg, (cards[None, :] - 1 - base).astype(np.uint16))


def test_discretize_constant_and_empty_columns():
    fit = np.array([[3.0, NAN], [3.0, NAN]])
    codes, cards = H.discretize(fit, [False, False], 2)
    assert cards.tolist() == [1, 0]
    assert codes.tolist() == [[0, 0xFFFF], [0, 0xFFFF]]


# ---- anti-contradiction filter (Section 4 preprocessing) --------------------

def test_filter_hand_example():
    rows = np.array([[1], [1], [1], [2], [2], [3], [1]], np.uint64)
    lab = np.array([1, 0, 1, 0, 0, 1, 0], np.uint8)
    # itemset {1}: attack at 0, 2; normal at 1, 6 -> pairs (0,1), (2,6): all dropped.
    # itemset {2}: normal only; {3}: attack only.
    assert H.filter_contradictions(rows, lab, 0).tolist() == [0, 0, 0, 1, 1, 1, 0]
    rows2 = np.array([[1], [1], [1], [5]], np.uint64)
    lab2 = np.array([0, 1, 1, 1], np.uint8)
    # {1}: normal 0, attack 1, 2 -> pair (1, 0) dropped, surplus attack 2 kept.
    assert H.filter_contradictions(rows2, lab2, 0).tolist() == [0, 0, 1, 1]
    assert H.filter_contradictions(rows2, lab2, 1).tolist() == [0, 0, 0, 1]


def test_filter_counts_brute_force():
    rng = np.random.default_rng(11)
    rows = rng.integers(0, 4, size=(200, 2)).astype(np.uint64)
    lab = rng.integers(0, 2, 200).astype(np.uint8)
    keep0 = H.filter_contradictions(rows, lab, 0)
    keep1 = H.filter_contradictions(rows, lab, 1)
    for key in {tuple(r) for r in rows.tolist()}:
        members = [i for i in range(200) if tuple(rows[i].tolist()) == key]
        a = [i for i in members if lab[i] == 1]
        n = [i for i in members if lab[i] == 0]
        k = min(len(a), len(n))
        assert sum(keep0[i] for i in a) == len(a) - k
        assert sum(keep0[i] for i in n) == len(n) - k
        # the survivors are the last ones in record order
        assert all(keep0[i] for i in a[k:]) and all(keep0[i] for i in n[k:])
        both = bool(a) and bool(n)
        assert all(keep1[i] != both for i in members)


# ---- metrics (Section 4, Table 2) ------------------------------------------

def test_confusion_hand_example():
    m = H.evaluate([1, 1, 0, 0, 1], [1, 0, 0, 1, 1])
    assert (m["tp"], m["fp"], m["tn"], m["fn"]) == (2, 1, 1, 1)
    assert m["accuracy"] == 3 / 5 and m["precision"] == 2 / 3
    assert m["recall"] == 2 / 3 and m["f1"] == 4 / 6
    assert math.isnan(m["auc"])
    # fp != fn, so precision and recall differ: tp 1, fp 3, tn 1, fn 2
    m = H.evaluate([1, 1, 1, 0, 0, 0, 0], [1, 0, 0, 1, 1, 1, 0])
    assert (m["tp"], m["fp"], m["tn"], m["fn"]) == (1, 3, 1, 2)
    assert m["accuracy"] == 2 / 7 and m["precision"] == 1 / 4
    assert m["recall"] == 1 / 3 and m["f1"] == 2 / 7
    e = H.evaluate([0, 0], [0, 0], [1, 2], [0, 0])
    assert math.isnan(e["precision"]) and math.isnan(e["recall"]) and math.isnan(e["auc"])


def test_auc_closed_forms():
    y = [1, 1, 0, 0]
    assert H.evaluate(y, y, [5, 6, 0, 1], [0, 0, 0, 0])["auc"] == 1.0
    assert H.evaluate(y, y, [0, 1, 5, 6], [0, 0, 0, 0])["auc"] == 0.0
    assert H.evaluate(y, y, [3, 3, 3, 3], [1, 1, 1, 1])["auc"] == 0.5
    # s = A - N: attack scores 2, 0; normal scores 0, -3
    # pairs (2,0) win, (2,-3) win, (0,0) tie, (0,-3) win -> (2+2+1+2) / 8
    assert H.evaluate(y, y, [2, 1, 4, 0], [0, 1, 4, 3])["auc"] == 7 / 8


def test_auc_matches_pairwise_brute_force():
    rng = np.random.default_rng(3)
    for trial in range(20):
        m = int(rng.integers(2, 60))
        y = rng.integers(0, 2, m)
        A = rng.integers(0, 6, m)
        N = rng.integers(0, 6, m)
        assert H.auc_two_u(y, A, N) == H.auc_brute(y, A, N)


def test_auc_matches_library_routine():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    y = rng.integers(0, 2, 3000)
    A = rng.integers(0, 50, 3000)
    N = rng.integers(0, 50, 3000)
    ours = H.evaluate(y, y, A, N)["auc"]
    assert abs(ours - sk.roc_auc_score(y, A - N)) < 1e-12


def test_reg3_sweep_matches_regulation_labels():
    rng = np.random.default_rng(8)
    A = rng.integers(0, 40, 500)
    N = rng.integers(0, 40, 500)
    A[:20] = 0
    N[:20] = 0
    y = rng.integers(0, 2, 500)
    mu, sigma = oracle.reg3_stats(N[y == 0])
    rs = [math.inf, 0.568, 0.0, -1.0, 2.0]
    out = H.reg3_sweep(A, N, y, mu, sigma, rs)
    for r, m in zip(rs, out):
        thr = None if math.isinf(r) else oracle.reg3_threshold(mu, sigma, r)
        lab = oracle.labels(A, N, thr)
        assert m == dict(H.evaluate(y, lab, A, N), r=r)
    # Regulation 3 only adds attack labels: recall cannot fall as r shrinks.
    assert out[2]["recall"] >= out[1]["recall"] >= out[0]["recall"]


def test_reg3_threshold_is_strict():
    # mu 10, sigma 2, r 1: threshold exactly 8.  N = 8 is not below it, so
    # the record (A 3 < N 8) stays normal; N = 7 turns attack.
    out = H.reg3_sweep([3, 3], [8, 7], [0, 1], 10.0, 2.0, [1.0])[0]
    assert (out["tn"], out["tp"], out["fp"], out["fn"]) == (1, 1, 0, 0)
