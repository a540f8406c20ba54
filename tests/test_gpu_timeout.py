"""Bounded device waits: a wait of the tensor-core kernel that runs out ends
the call with IG_E_TIMEOUT, and the process goes on to fit and score exactly.

The library's test hook IG_TEST_STALL_UNIT=u makes every CTA of the fused
tensor-core kernel wait, before the MMAs of its u-th unit, on a barrier that
nothing ever arrives on, with its stage and accumulator waits cut to a few
polls.  The kernel then records the timeout, drains the copies and MMAs it
has in flight (those waits keep their full limit), frees its tensor memory
and ends; the host reads the status word and reports IG_E_TIMEOUT.  No GPU
fault, trap or endless wait is involved: every wait is bounded.
"""
import numpy as np
import pytest

import igdata
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_14222_gb300 as ig  # noqa: E402

IG_E_TIMEOUT = -4


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    w = igdata.tiny()
    rows = ig.ig_encode(torch.from_numpy(w.train_codes.view(np.int16)).cuda(), w.cards)
    labels = torch.from_numpy(w.train_labels).cuda()
    test = ig.ig_encode(torch.from_numpy(w.test_codes.view(np.int16)).cuda(), w.cards)
    om = oracle.fit(oracle.encode(w.train_codes, w.cards), w.train_labels)
    want = oracle.score(om, oracle.encode(w.test_codes, w.cards))
    return rows, labels, test, om, want


def _assert_exact(m, om, test, want):
    for cls in (0, 1):
        words, f, s = m.patterns(cls)
        assert np.array_equal(words, om.patterns[cls])
        assert np.array_equal(f, om.support[cls]) and np.array_equal(s, om.score[cls])
    A, N, lab = ig.ig_score(m, test)
    for got, exp in zip((A, N, lab), want):
        assert np.array_equal(got.cpu().numpy(), exp)


@pytest.mark.parametrize("stall_unit", [0, 1])
def test_fit_timeout_then_exact_fit(tiny, monkeypatch, stall_unit):
    # Unit 0: the kernel stops before any MMA; unit 1: with the first
    # unit's MMAs issued, which the drain must wait for.
    rows, labels, test, om, want = tiny
    monkeypatch.setenv("IG_TEST_STALL_UNIT", str(stall_unit))
    with pytest.raises(ig.IGError) as e:
        ig.ig_fit(rows, labels, subset_kernel=4)
    assert e.value.code == IG_E_TIMEOUT
    monkeypatch.delenv("IG_TEST_STALL_UNIT")
    _assert_exact(ig.ig_fit(rows, labels, subset_kernel=4), om, test, want)


def test_score_timeout_then_exact_score(tiny, monkeypatch):
    # The evidence launch (Eq. 4, patterns resident) stalls at its second
    # unit; the same model then scores exactly.
    rows, labels, test, om, want = tiny
    m = ig.ig_fit(rows, labels, subset_kernel=4)
    assert test.shape[0] >= 512            # large enough for the item index
    monkeypatch.setenv("IG_TEST_STALL_UNIT", "1")
    with pytest.raises(ig.IGError) as e:
        ig.ig_score(m, test)
    assert e.value.code == IG_E_TIMEOUT
    monkeypatch.delenv("IG_TEST_STALL_UNIT")
    _assert_exact(m, om, test, want)
