"""Serving: patterns given from outside, the continuous-batching server, and
the batched fit -- all against ig_score / ig_fit and the CPU oracle.
"""
import threading
import time

import numpy as np
import pytest

import igdata
import oracle
from tests import golden_digests

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_14222_gb300 as ig  # noqa: E402


@pytest.fixture(scope="module")
def served():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    sw = igdata.served(per_class=30000, total_flows=24000, seed=77)
    words = [ig.ig_encode(sw.patterns[c], sw.cards) for c in (0, 1)]   # host path
    model = ig.ig_model_from_patterns(words[0], sw.support[0], words[1], sw.support[1])
    flows = ig.ig_encode(sw.flow_codes, sw.cards)
    return sw, words, model, flows


def test_model_from_patterns_matches_oracle(served):
    # The oracle's model is built from the generator's codes alone (its own
    # encoding, canonical order and Eq. 2 scores); so are the test records.
    sw, words, model, flows = served
    om = oracle.model_from_patterns({c: oracle.encode(sw.patterns[c], sw.cards) for c in (0, 1)},
                                    sw.support)
    for c in (0, 1):
        w, f, s = model.patterns(c)
        assert np.array_equal(w, om.patterns[c])
        assert np.array_equal(f, om.support[c]) and np.array_equal(s, om.score[c])
    test = oracle.encode(sw.flow_codes[:3000], sw.cards)
    A, N, lab = ig.ig_score(model, test)
    oA, oN, olab = oracle.score(om, test)
    assert np.array_equal(A, oA) and np.array_equal(N, oN) and np.array_equal(lab, olab)


def test_served_full_size(served):
    # The served workload at its full size: 1M normal + 1M attack patterns,
    # 10^6 flows in 1,972 requests.  The one-shot ig_score of a seeded
    # sample of flows equals the oracle's; the model and the one-shot
    # ig_score of all flows equal the oracle's digest of the same workload;
    # every flow the server returns, in a burst of all requests at once,
    # equals the one-shot ig_score of all flows.
    sw = igdata.served()
    words = [ig.ig_encode(torch.from_numpy(sw.patterns[c].view(np.int16)).cuda(), sw.cards)
             for c in (0, 1)]
    model = ig.ig_model_from_patterns(words[0], sw.support[0], words[1], sw.support[1])
    om = oracle.model_from_patterns({c: oracle.encode(sw.patterns[c], sw.cards) for c in (0, 1)},
                                    sw.support)
    idx = np.random.default_rng(9).choice(sw.flow_codes.shape[0], 1500, replace=False)
    sample = oracle.encode(sw.flow_codes[idx], sw.cards)
    A, N, lab = ig.ig_score(model, sample)
    oA, oN, olab = oracle.score(om, sample)
    assert np.array_equal(A, oA) and np.array_equal(N, oN) and np.array_equal(lab, olab)
    assert int((oA > 0).sum()) > 0 and int((oN > 0).sum()) > 0
    flows = ig.ig_encode(sw.flow_codes, sw.cards)
    ref = ig.ig_score(model, flows)
    want = golden_digests.stored()[sw.name]
    info = model.info()
    pats = {c: model.patterns(c) for c in (0, 1)}
    got = golden_digests.writer().digest(
        info["n_candidates"], {c: pats[c][0] for c in (0, 1)}, {c: pats[c][1] for c in (0, 1)},
        {c: pats[c][2] for c in (0, 1)}, ref[0], ref[1], ref[2])
    assert list(info["n_patterns"]) == want["n_patterns"]
    assert got == want["sha256"], "served output differs from the oracle's"
    offs = np.concatenate([[0], np.cumsum(sw.request_sizes)])
    reqs = [flows[offs[i]:offs[i + 1]] for i in range(len(sw.request_sizes))]
    outs, (batches, n_flows) = _serve(model, reqs, 0.0, cap=65536, budget=1 << 30)
    assert n_flows == flows.shape[0] and batches < len(reqs)
    for k in range(3):
        assert np.array_equal(np.concatenate([o[k] for o in outs]), ref[k])


def test_model_from_patterns_rejects_duplicates():
    rows = np.array([[3], [5], [3]], np.uint64)
    with pytest.raises(ig.IGError) as e:
        ig.ig_model_from_patterns(rows, np.ones(3, np.uint32), rows[:1], np.ones(1, np.uint32))
    assert e.value.code == -1


@pytest.mark.parametrize("rows", [7, 900])   # dense (small batch) and item-index scoring
def test_small_and_large_batches_agree(served, rows):
    sw, words, model, flows = served
    A, N, lab = ig.ig_score(model, flows[:rows])
    A2, N2, lab2 = ig.ig_score(model, torch.from_numpy(flows[:rows].view(np.int64)).cuda())
    assert np.array_equal(A, A2.cpu().numpy()) and np.array_equal(N, N2.cpu().numpy())
    assert np.array_equal(lab, lab2.cpu().numpy())


def _serve(model, reqs, pause_s, slots=3, cap=8192, budget=64 << 20):
    server = ig.Server(model, slots=slots, max_batch_flows=cap, memory_budget_bytes=budget)
    tickets = []

    def submit_all():
        for r in reqs:
            tickets.append(server.submit(r))
            if pause_s:
                time.sleep(pause_s)
    th = threading.Thread(target=submit_all)
    th.start()
    th.join()
    outs = [server.wait(t) for t in tickets]
    stats = server.stats()
    server.close()
    return outs, stats


@pytest.mark.parametrize("pause_s", [0.0, 0.0003], ids=["burst", "paced"])
def test_server_results_same_alone_and_in_the_mix(served, pause_s):
    sw, words, model, flows = served
    refA, refN, reflab = ig.ig_score(model, flows)
    offs = np.concatenate([[0], np.cumsum(sw.request_sizes)])
    reqs = [flows[offs[i]:offs[i + 1]] for i in range(len(sw.request_sizes))]
    outs, (batches, scored) = _serve(model, reqs, pause_s)
    assert scored == flows.shape[0]
    if pause_s == 0.0:
        assert batches < len(reqs)                # a burst is batched together
    for i, (A, N, lab, ms) in enumerate(outs):
        sl = slice(offs[i], offs[i + 1])
        assert np.array_equal(A, refA[sl]) and np.array_equal(N, refN[sl])
        assert np.array_equal(lab, reflab[sl])
        assert ms >= 0
    # Alone: a request scored by itself gives the same numbers.
    for i in (0, len(reqs) // 2, len(reqs) - 1):
        A, N, lab = ig.ig_score(model, reqs[i])
        assert np.array_equal(A, outs[i][0]) and np.array_equal(lab, outs[i][2])


def test_server_memory_admission(served):
    # A budget of a few requests' worth still serves everything, exactly.
    sw, words, model, flows = served
    offs = np.concatenate([[0], np.cumsum(sw.request_sizes)])
    reqs = [flows[offs[i]:offs[i + 1]] for i in range(len(sw.request_sizes))]
    outs, (batches, scored) = _serve(model, reqs, 0.0, budget=4096 * 9000)
    refA, _, reflab = ig.ig_score(model, flows)
    assert scored == flows.shape[0]
    assert np.array_equal(np.concatenate([o[0] for o in outs]), refA)
    assert np.array_equal(np.concatenate([o[2] for o in outs]), reflab)


def test_autotuner_choices_keep_results(tmp_path):
    from paper_2507_14222_gb300 import autotune
    probs = igdata.batched(6)
    enc = []
    for w in probs:
        codes = torch.from_numpy(w.train_codes.view(np.int16)).cuda()
        tests = torch.from_numpy(w.test_codes.view(np.int16)).cuda()
        enc.append((ig.ig_encode(codes, w.cards), torch.from_numpy(w.train_labels).cuda(),
                    ig.ig_encode(tests, w.cards)))
    tuner = autotune.Autotuner(str(tmp_path / "tune.json"))
    chosen = tuner.tune(enc, repeats=1)
    assert chosen and all(c in autotune.CANDIDATES for c in chosen.values())
    assert (tmp_path / "tune.json").exists()
    again = autotune.Autotuner(str(tmp_path / "tune.json"))     # read back from the cache
    params = [again.params_for(int(r.shape[1]), int(r.shape[0])) for r, _, _ in enc]
    assert all(p is not None for p in params)
    tuned = ig.ig_fit_batched([(r, lab) for r, lab, _ in enc], per_problem_params=params)
    for (r, lab, t), mt in zip(enc, tuned):
        plain = ig.ig_fit(r, lab)
        for cls in (0, 1):
            assert all(np.array_equal(x, y) for x, y in zip(mt.patterns(cls), plain.patterns(cls)))
        a1 = ig.ig_score(mt, t)
        a2 = ig.ig_score(plain, t)
        assert all(torch.equal(x, y) for x, y in zip(a1, a2))


@pytest.mark.parametrize("cfg", [dict(index_max_q=1), dict(index_max_q=2),
                                 dict(index_flip_factor=1), dict(index_flip_factor=1 << 20)])
def test_index_tiling_knobs_keep_results(cfg):
    w = igdata.nsl15k()
    rows = ig.ig_encode(torch.from_numpy(w.train_codes.view(np.int16)).cuda(), w.cards)
    lab = torch.from_numpy(w.train_labels).cuda()
    test = ig.ig_encode(torch.from_numpy(w.test_codes.view(np.int16)).cuda(), w.cards)
    base = ig.ig_fit(rows, lab)
    tuned = ig.ig_fit(rows, lab, **cfg)
    for cls in (0, 1):
        assert all(np.array_equal(x, y) for x, y in zip(tuned.patterns(cls), base.patterns(cls)))
    assert all(torch.equal(x, y) for x, y in zip(ig.ig_score(tuned, test), ig.ig_score(base, test)))
