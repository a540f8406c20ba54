"""The autotuner's host logic (no GPU): grouping of problems, choice of the
fastest candidate per group, and the cache that makes tuning once per
machine.  The fit and the clock are replaced by fakes; only the tuner's
bookkeeping runs."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2507_14222_gb300 as ig  # noqa: E402
from paper_2507_14222_gb300 import autotune  # noqa: E402


def test_bucket_groups_by_word_power_of_two_and_log2_records():
    assert autotune.bucket(8, 3000) == "kt8-n2^12"
    assert autotune.bucket(7, 3000) == "kt8-n2^12"      # K rounds up to a power of two
    assert autotune.bucket(9, 3000) == "kt16-n2^12"
    assert autotune.bucket(1, 1) == "kt1-n2^0"
    assert autotune.bucket(4, 5800) == "kt4-n2^13"      # log2 rounded to the nearest


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def perf_counter(self):
        return self.t


def problem(n, K):
    rows = np.zeros((n, K), np.uint64)
    return rows, np.zeros(n, np.uint8), rows[: max(1, n // 10)]


@pytest.fixture
def fake_fit(monkeypatch):
    """ig_fit costs 1 + (position of its configuration in a ranking) time
    units, the ranking depending on the group, so that each group has a
    different fastest choice."""
    clock = FakeClock()
    calls = []
    ranking = {8: [{"subset_kernel": 4}, {"subset_kernel": 2}],
               4: [{"subset_kernel": 1}, {"subset_kernel": 4}]}

    class Model:
        def free(self):
            pass

    def fit(rows, labels, **cfg):
        K = rows.shape[1]
        order = ranking[K]
        cost = order.index(cfg) + 1 if cfg in order else 10
        clock.t += cost
        calls.append((K, json.dumps(cfg, sort_keys=True), rows.shape[0]))
        return Model()

    monkeypatch.setattr(ig, "ig_fit", fit)
    monkeypatch.setattr(ig, "ig_score", lambda model, test: None)
    monkeypatch.setattr(autotune.time, "perf_counter", clock.perf_counter)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(autotune.Autotuner, "_device_key", staticmethod(lambda: "FakeGPU/152sm"))
    return calls


def test_tune_picks_fastest_per_group_and_caches(tmp_path, fake_fit):
    cands = [{"subset_kernel": 2}, {"subset_kernel": 4}, {"subset_kernel": 1}]
    probs = [problem(3000, 8), problem(2900, 8), problem(3100, 4)]
    path = str(tmp_path / "tune.json")
    chosen = autotune.Autotuner(path).tune(probs, candidates=cands, repeats=1)
    assert chosen == {"FakeGPU/152sm/kt8-n2^12": {"subset_kernel": 4},
                      "FakeGPU/152sm/kt4-n2^12": {"subset_kernel": 1}}
    # One representative per group, every candidate timed (warm-up + repeats).
    assert len(fake_fit) == 2 * len(cands) * 2
    with open(path) as f:
        assert json.load(f) == chosen

    # A second tuner reads the cache and times nothing for known groups.
    fake_fit.clear()
    again = autotune.Autotuner(path)
    assert again.tune(probs, candidates=cands, repeats=1) == chosen
    assert fake_fit == []
    assert again.config_for(8, 3000) == {"subset_kernel": 4}
    assert again.config_for(16, 3000) is None

    # retune=True times them again.
    again.tune(probs, candidates=cands, repeats=1, retune=True)
    assert len(fake_fit) == 2 * len(cands) * 2


def test_representative_is_the_median_sized_problem(tmp_path, fake_fit):
    probs = [problem(3300, 8), problem(2900, 8), problem(3000, 8)]   # one group: n ~ 2^12
    autotune.Autotuner(str(tmp_path / "t.json")).tune(
        probs, candidates=[{"subset_kernel": 4}], repeats=1)
    assert [n for _, _, n in fake_fit] == [3000, 3000]   # the median, warm-up + one repeat
