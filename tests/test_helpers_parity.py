"""The library's host helpers (include/ig_helpers.h) against the oracle, bit
for bit, on seeded inputs.  The helpers are host code, so these run on the
CPU through the C ABI; no GPU is involved."""
import math
import shutil
import os

import numpy as np
import pytest

import igdata
import paper_2507_14222_gb300 as ig
from oracle import helpers as H

pytestmark = pytest.mark.skipif(
    not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")),
    reason="nvcc not available to build the library")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ig.build()
    ig.load()


def _same_metrics(a: dict, b: dict):
    assert a.keys() == b.keys()
    for k in a:
        x, y = a[k], b[k]
        if isinstance(x, float) and math.isnan(x):
            assert isinstance(y, float) and math.isnan(y), k
        else:
            assert x == y, (k, x, y)


@pytest.mark.parametrize("p", [0, 1, 2])
def test_discretize_matches_oracle(p):
    raw = igdata.raw_flows(3000, seed=1006)
    fit, test = raw.values[:2000], raw.values[2000:]
    codes, cards = ig.ig_discretize(fit, raw.categorical, p)
    o_codes, o_cards = H.discretize(fit, raw.categorical, p)
    assert np.array_equal(cards, o_cards)
    assert np.array_equal(codes, o_codes)
    t_codes, t_cards = ig.ig_discretize(fit, raw.categorical, p, values=test)
    o_t, _ = H.discretize(fit, raw.categorical, p, values=test)
    assert np.array_equal(t_cards, o_cards)
    assert np.array_equal(t_codes, o_t)
    # Every missing entry of the fit rows is coded missing, nothing else is.
    assert np.array_equal(codes == 0xFFFF, ~np.isfinite(fit))


def test_discretize_edge_cases():
    nan, inf = float("nan"), float("inf")
    fit = np.array([[3.0, nan, -0.0, 1.0], [3.0, nan, 0.0, inf], [3.0, nan, 2.0, 5.0]])
    cat = np.array([0, 0, 1, 0], np.uint8)
    got = ig.ig_discretize(fit, cat, 3)
    want = H.discretize(fit, cat, 3)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert got[1].tolist() == [1, 0, 2, 2]
    # no rows at all
    empty = np.zeros((0, 4))
    c, k = ig.ig_discretize(empty, cat, 0)
    assert c.shape == (0, 4) and k.tolist() == [0, 0, 0, 0]


def test_discretize_rejects_bad_arguments():
    fit = np.zeros((3, 2))
    with pytest.raises(ig.IGError) as e:
        ig.ig_discretize(fit, [0, 0], 10)
    assert e.value.code == -1          # IG_E_INVAL
    many = np.arange(70000, dtype=float).reshape(-1, 1)
    with pytest.raises(ig.IGError) as e:
        ig.ig_discretize(many, [1], 0)
    assert e.value.code == -5          # IG_E_OVERFLOW: more than 65535 tokens


def test_pipeline_codes_feed_the_encoder_shape():
    # Discretised codes are valid ig_encode input: code < card or missing.
    raw = igdata.raw_flows(1000, seed=7)
    codes, cards = ig.ig_discretize(raw.values, raw.categorical, 0)
    ok = (codes < cards[None, :].astype(np.int64)) | (codes == 0xFFFF)
    assert ok.all()


@pytest.mark.parametrize("mode", [0, 1])
def test_filter_matches_oracle(mode):
    rng = np.random.default_rng(21 + mode)
    for K, n, spread in ((1, 500, 6), (3, 2000, 4), (8, 3000, 40)):
        rows = rng.integers(0, spread, size=(n, K)).astype(np.uint64)
        rows[:, 0] |= np.uint64(1) << np.uint64(63)     # high bits in play
        lab = rng.integers(0, 2, n).astype(np.uint8)
        got = ig.ig_filter_contradictions(rows, lab, mode)
        assert np.array_equal(got, H.filter_contradictions(rows, lab, mode))


def test_filter_edge_cases():
    rows = np.zeros((0, 2), np.uint64)
    assert ig.ig_filter_contradictions(rows, np.zeros(0, np.uint8)).shape == (0,)
    rows = np.ones((5, 1), np.uint64)
    assert ig.ig_filter_contradictions(rows, np.ones(5, np.uint8)).all()
    with pytest.raises(ig.IGError):
        ig.ig_filter_contradictions(rows, np.full(5, 2, np.uint8))
    with pytest.raises(ig.IGError):
        ig.ig_filter_contradictions(rows, np.ones(5, np.uint8), mode=2)


def test_filter_on_encoded_workload():
    # The stand-in for the 15k NSL-KDD slice, one-hot encoded (K = 8).
    import oracle
    w = igdata.nsl15k()
    rows = oracle.encode(w.train_codes, w.cards)
    for mode in (0, 1):
        got = ig.ig_filter_contradictions(rows, w.train_labels, mode)
        assert np.array_equal(got, H.filter_contradictions(rows, w.train_labels, mode))


def test_evaluate_matches_oracle():
    rng = np.random.default_rng(31)
    for m, hi in ((1, 3), (2, 3), (57, 4), (5000, 30), (20000, 10 ** 12)):
        y = rng.integers(0, 2, m).astype(np.uint8)
        yp = rng.integers(0, 2, m).astype(np.uint8)
        A = rng.integers(0, hi, m)
        N = rng.integers(0, hi, m)
        _same_metrics(ig.ig_evaluate(y, yp, A, N), H.evaluate(y, yp, A, N))
        _same_metrics(ig.ig_evaluate(y, yp), H.evaluate(y, yp))
    # extremes of the int64 evidence range
    big = np.array([2 ** 62, 0, 2 ** 63 - 1, 5], np.int64)
    y = np.array([1, 0, 1, 0], np.uint8)
    _same_metrics(ig.ig_evaluate(y, y, big, big[::-1].copy()),
                  H.evaluate(y, y, big, big[::-1].copy()))
    _same_metrics(ig.ig_evaluate(np.zeros(0, np.uint8), np.zeros(0, np.uint8)),
                  H.evaluate([], []))


def test_reg3_sweep_matches_oracle():
    rng = np.random.default_rng(41)
    m = 4000
    A = rng.integers(0, 200, m)
    N = rng.integers(0, 200, m)
    A[:50] = 0
    N[:50] = 0
    y = rng.integers(0, 2, m).astype(np.uint8)
    mu, sigma = float(N.mean()), float(N.std())
    rs = [math.inf, 2.0, 0.568, 0.0, -0.5, -3.0]
    got = ig.ig_reg3_sweep(A, N, y, mu, sigma, rs)
    want = H.reg3_sweep(A, N, y, mu, sigma, rs)
    for g, w in zip(got, want):
        _same_metrics(g, w)
    # sigma 0 with r = inf: the threshold is NaN, Regulation 3 never fires
    got = ig.ig_reg3_sweep(A, N, y, 5.0, 0.0, [math.inf])
    _same_metrics(got[0], H.reg3_sweep(A, N, y, 5.0, 0.0, [math.inf])[0])
