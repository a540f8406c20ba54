"""The stage profiler (ig_prof_*): totals, timeline and launch counts agree
with one another on a real fit and score.  Timing only -- no results are
checked here (the parity tests do that)."""
import numpy as np
import pytest

import igdata

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_14222_gb300 as ig  # noqa: E402


@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    w = igdata.nsl_like(3000, 0.5, 4242, "profiler-3k")
    rows = ig.ig_encode(torch.from_numpy(w.train_codes.view(np.int16)).cuda(), w.cards)
    test = ig.ig_encode(torch.from_numpy(w.test_codes.view(np.int16)).cuda(), w.cards)
    labels = torch.from_numpy(w.train_labels).cuda()
    return rows, labels, test


def test_timeline_matches_stage_totals(workload):
    rows, labels, test = workload
    ig.prof_reset()
    ig.prof_enable(True)
    launches0 = ig.launch_count()
    model = ig.ig_fit(rows, labels)
    ig.ig_score(model, test)
    torch.cuda.synchronize()
    ig.prof_enable(False)
    launched = ig.launch_count() - launches0
    spans = ig.prof_timeline()
    totals = ig.prof_read()
    model.free()
    names = {name for name, *_ in spans}
    assert {"pair_insert", "compact", "canonical_sort"} <= names
    assert all(t1 >= t0 >= 0.0 for _, _, t0, t1 in spans)
    # Every stage's spans add up to its total, and there is one span per timed launch.
    for name, (ms, n, _work) in totals.items():
        mine = [t1 - t0 for s, _, t0, t1 in spans if s == name]
        assert len(mine) == n, name
        assert abs(sum(mine) - ms) <= 1e-3 * max(1.0, ms), name
    # The library launched at least one kernel per recorded span.
    assert launched >= len(spans) > 0
    # The two classes ran on two streams besides the caller's.
    assert len({sid for _, sid, _, _ in spans}) >= 3


def test_reset_clears_the_timeline(workload):
    rows, labels, _ = workload
    ig.prof_reset()
    ig.prof_enable(True)
    ig.ig_fit(rows, labels).free()
    torch.cuda.synchronize()
    ig.prof_enable(False)
    assert len(ig.prof_timeline()) > 0
    ig.prof_reset()
    assert ig.prof_timeline() == []
    assert all(n == 0 for _, n, _ in ig.prof_read().values())


def test_select_times_only_the_chosen_stage(workload):
    rows, labels, test = workload
    ig.prof_select(["pair_insert"])
    try:
        ig.prof_reset()
        ig.prof_enable(True)
        model = ig.ig_fit(rows, labels)
        ig.ig_score(model, test)
        torch.cuda.synchronize()
        ig.prof_enable(False)
        totals = ig.prof_read()
        model.free()
    finally:
        ig.prof_select(None)
    timed = {name for name, (_ms, n, _w) in totals.items() if n}
    assert timed == {"pair_insert"}
    assert totals["pair_insert"][1] >= 2  # at least one launch per class
    # Executed-test counts are kept for unselected stages too.
    assert any(w > 0 for name, (_ms, _n, w) in totals.items() if name != "pair_insert")
