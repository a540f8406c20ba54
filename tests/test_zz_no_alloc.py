"""ig_score_noalloc: scoring without any device allocation inside the library.

The entry point exists for callers that cannot let the library allocate
device memory for them -- a latency-bound flow-scoring loop where an
allocation could stall or fail under memory pressure, or a process whose
device memory is reserved up front by another allocator.  Its scratch lives
in one fixed device array inside the library, shared by every call, so this
test checks two calls in a row (different records each time, so stale
contents of the shared array would show) against ig_score, exactly: A, N and
the labels are integers.

Collected last on purpose (file name) and self-contained: it fits its own
model, so it passes alone in a fresh process as well as after the others.
"""
import ctypes

import numpy as np
import pytest

import igdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_14222_gb300 as ig  # noqa: E402


@pytest.fixture(scope="module")
def model_and_rows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    w = igdata.tiny()
    rows = ig.ig_encode(torch.from_numpy(w.train_codes.view(np.int16)).cuda(), w.cards)
    model = ig.ig_fit(rows, torch.from_numpy(w.train_labels).cuda())
    test = ig.ig_encode(torch.from_numpy(w.test_codes.view(np.int16)).cuda(), w.cards)
    return model, test, rows


def test_two_calls_match_ig_score(model_and_rows):
    model, test, train_rows = model_and_rows
    for rows in (test, train_rows[:377]):          # two calls in a row
        A, N, lab = ig.ig_score_noalloc(model, rows)
        rA, rN, rlab = ig.ig_score(model, rows)
        torch.cuda.synchronize()
        assert torch.equal(A, rA) and torch.equal(N, rN) and torch.equal(lab, rlab)
        assert int((A > 0).sum()) > 0                # the check is not vacuous


def test_limits_are_rejected(model_and_rows):
    model, test, _ = model_and_rows
    lib = ig.load()
    too_many = ig.SCORE_NOALLOC_MAX_ROWS + 1
    rc = lib.ig_score_noalloc(model.handle, ctypes.c_void_p(test.data_ptr()), too_many,
                              None, None, None, None)
    assert rc == -1 and b"IG_SCORE_NOALLOC_MAX_ROWS" in lib.ig_last_error()
    host_rows = test.cpu().numpy()
    rc = lib.ig_score_noalloc(model.handle, ctypes.c_void_p(host_rows.ctypes.data),
                              host_rows.shape[0], None, None, None, None)
    assert rc == -1 and b"device memory" in lib.ig_last_error()


@pytest.mark.parametrize("n_items", [150, 300, 420])   # K = 3, 5, 7: row stride < padded width
def test_odd_word_counts_match_oracle(n_items):
    # A record of K words is read with its own stride K while the kernels
    # work on the padded width (4 or 8 words); the words past K must read
    # as zero.  Two calls in a row again, against the CPU oracle.
    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    rng = np.random.default_rng(n_items)
    rows = igdata.random_words(rng, 260, n_items, "three_quarters")
    labels = np.zeros(260, np.uint8)
    labels[rng.permutation(260)[:120]] = 1
    model = ig.ig_fit(torch.from_numpy(rows.view(np.int64)).cuda(),
                      torch.from_numpy(labels).cuda())
    om = oracle.fit(rows, labels)
    # Random records (mostly no pattern inside) and training records (their
    # own patterns inside), a different mix in each call.
    for test in (np.concatenate([igdata.random_words(rng, 200, n_items, "three_quarters"),
                                 rows[:133]]),
                 rows[130:221]):
        A, N, lab = ig.ig_score_noalloc(model, torch.from_numpy(test.view(np.int64)).cuda())
        oA, oN, olab = oracle.score(om, test)
        assert np.array_equal(A.cpu().numpy(), oA) and np.array_equal(N.cpu().numpy(), oN)
        assert np.array_equal(lab.cpu().numpy(), olab)
        assert int((A > 0).sum()) + int((N > 0).sum()) > 0


def test_width_mismatch_rejected_before_launch(model_and_rows):
    model, test, _ = model_and_rows
    launches = ig.launch_count()
    with pytest.raises(ValueError, match="words per record"):
        ig.ig_score_noalloc(model, test[:, :2].contiguous())
    with pytest.raises(ValueError, match="64-bit words"):
        ig.ig_score_noalloc(model, test.to(torch.int32))
    with pytest.raises(ValueError, match="words per record"):
        ig.ig_score(model, test[:, :3].contiguous())
    assert ig.launch_count() == launches
