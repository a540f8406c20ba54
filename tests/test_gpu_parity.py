"""CUDA library vs CPU oracle, element by element (all integer: bit-exact).

Covers the C ABI end to end -- ig_encode, ig_fit, ig_score, persistence --
on the seeded workloads (500-record, 15k and 148k NSL-KDD-shaped), random
dense itemsets of every word count K in 1..16 with ragged sizes around the
64-record pair tile, brute-force tiny cases, and the degenerate cases of the
method (identical classes, disjoint classes, a single record per class,
duplicate records, empty intersections, an empty class).
"""
import os

import numpy as np
import pytest

import igdata
import oracle
from tests import brute
from tests import golden_digests

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_14222_gb300 as ig  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ig.build()
    ig.load()


def dev(a):
    """numpy -> CUDA tensor holding the same bytes."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint16:
        a = a.view(np.int16)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


# 1 = integer-pipe (LOP3) kernel, 2 = tensor-core (tcgen05) kernel,
# 3 = item-index pruning (exact)
KERNELS = [1, 2, 3, 4]


def gpu_fit(rows, labels, r=None, kernel=0):
    return ig.ig_fit(dev(rows), dev(np.asarray(labels, np.uint8)), r=r, subset_kernel=kernel)


def assert_model_equal(m, om):
    info = m.info()
    for cls in (0, 1):
        words, f, s = m.patterns(cls)
        want = om.patterns[cls]
        assert words.shape == want.shape, (cls, words.shape, want.shape)
        assert np.array_equal(words, want), f"class {cls}: pattern sets differ"
        assert np.array_equal(f, om.support[cls]), f"class {cls}: supports differ"
        assert np.array_equal(s, om.score[cls]), f"class {cls}: scores differ"
        assert info["n_candidates"][cls] == om.n_candidates[cls]


_ORACLE_CACHE = {}


def _oracle_fit_cached(key, rows, labels):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.fit(rows, labels)
    return _ORACLE_CACHE[key]


def assert_scores_equal(m, om, rows):
    A, N, lab = ig.ig_score(m, dev(rows))
    oA, oN, olab = oracle.score(om, rows)
    assert np.array_equal(host(A, np.int64), oA)
    assert np.array_equal(host(N, np.int64), oN)
    assert np.array_equal(host(lab, np.uint8), olab)


# ---- encoding ---------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "nsl15k"])
def test_encode_parity(name):
    w = igdata.WORKLOADS[name]()
    for codes in (w.train_codes, w.test_codes):
        got = ig.ig_encode(dev(codes), w.cards)
        assert np.array_equal(host(got, np.uint64), oracle.encode(codes, w.cards))


def test_encode_ragged_and_wide():
    rng = np.random.default_rng(3)
    cards = rng.integers(1, 40, size=37).astype(np.uint16)   # L not a multiple of 64
    codes = np.stack([rng.integers(0, c, size=129) for c in cards], 1).astype(np.uint16)
    got = ig.ig_encode(dev(codes), cards)
    assert np.array_equal(host(got, np.uint64), oracle.encode(codes, cards))
    empty = ig.ig_encode(dev(codes[:0]), cards)
    assert tuple(empty.shape) == (0, (int(cards.astype(int).sum()) + 63) // 64)


def test_encode_missing_values():
    rng = np.random.default_rng(4)
    cards = np.array([16] * 32, np.uint16)
    codes = rng.integers(0, 16, size=(300, 32)).astype(np.uint16)
    codes[rng.random(codes.shape) < 0.4] = 0xFFFF
    got = ig.ig_encode(dev(codes), cards)
    assert np.array_equal(host(got, np.uint64), oracle.encode(codes, cards))


def test_encode_rejects_out_of_range_code():
    codes = np.array([[0, 1], [2, 5]], np.uint16)
    with pytest.raises(ig.IGError) as e:
        ig.ig_encode(dev(codes), [3, 5])
    assert e.value.code == -1


# ---- fit and score on brute-force and random cases --------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("seed", range(10))
def test_fit_against_brute_force(seed, kernel):
    rng = np.random.default_rng(100 + seed)
    L = 12
    K, positions = (1, list(range(L))) if seed % 2 else (2, list(range(58, 58 + L)))
    pool = [int(v) for v in rng.integers(1, 1 << L, size=7)]
    XA = [pool[i] for i in rng.integers(0, 7, size=3 + seed)]
    XN = [pool[i] for i in rng.integers(0, 7, size=2 + (seed * 3) % 7)]
    want = brute.fit(XA, XN, L)
    rows = np.concatenate([brute.pack(XA, positions, K), brute.pack(XN, positions, K)])
    labels = np.array([1] * len(XA) + [0] * len(XN), np.uint8)
    m = gpu_fit(rows, labels, kernel=kernel)
    for cls in (0, 1):
        words, f, s = m.patterns(cls)
        B, P, ff, S = want[cls]
        assert np.array_equal(words, brute.pack(P, positions, K).reshape(-1, K))
        assert f.tolist() == ff and s.tolist() == S
        assert m.info()["n_candidates"][cls] == len(B)
    tests = list(range(0, 1 << L, 5))
    A, N, lab = ig.ig_score(m, dev(brute.pack(tests, positions, K)))
    for i, t in enumerate(tests):
        a = brute.evidence(want[1][1], want[1][3], t)
        n = brute.evidence(want[0][1], want[0][3], t)
        assert (int(A[i]), int(N[i]), int(lab[i])) == (a, n, brute.label(a, n))


RANDOM_CASES = [
    # (n_items, n_attack, n_normal, density, duplicate pool or 0)
    (40, 1, 1, "half", 0),
    (64, 2, 3, "half", 0),
    (70, 63, 65, "three_quarters", 0),
    (128, 64, 64, "half", 0),
    (150, 65, 129, "three_quarters", 12),
    (250, 130, 70, "three_quarters", 0),
    (300, 200, 190, "half", 40),
    (520, 129, 63, "three_quarters", 0),
    (600, 100, 90, "three_quarters", 0),
    (1024, 150, 140, "three_quarters", 20),
    (1000, 70, 80, "three_quarters", 0),
    (256, 700, 650, "three_quarters", 0),    # > 512 per class: last coherence window
    (500, 600, 900, "three_quarters", 30),
    (256, 300, 280, "eighth", 0),            # sparse: the item index is used
    (512, 260, 400, "eighth", 25),
    (1024, 200, 150, "eighth", 0),
]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", RANDOM_CASES, ids=lambda c: f"L{c[0]}-{c[1]}x{c[2]}")
def test_fit_and_score_random(case, kernel):
    L, na, nn, density, pool = case
    rng = np.random.default_rng(L * 7 + na)
    if pool:
        base = igdata.random_words(rng, pool, L, density)
        rows = base[rng.integers(0, pool, size=na + nn)]
    else:
        rows = igdata.random_words(rng, na + nn, L, density)
    labels = np.zeros(na + nn, np.uint8)
    labels[rng.permutation(na + nn)[:na]] = 1
    m = gpu_fit(rows, labels, kernel=kernel)
    om = _oracle_fit_cached(case, rows, labels)
    assert_model_equal(m, om)
    test = igdata.random_words(rng, 97, L, "three_quarters")
    assert_scores_equal(m, om, np.concatenate([test, rows]))


def test_identical_classes():
    rng = np.random.default_rng(11)
    X = igdata.random_words(rng, 40, 200, "half")
    rows = np.concatenate([X, X[::-1]])
    labels = np.array([1] * 40 + [0] * 40, np.uint8)
    m = gpu_fit(rows, labels)
    assert m.info()["n_patterns"] == (0, 0)
    A, N, lab = ig.ig_score(m, dev(rows))
    assert int(A.abs().sum()) == 0 and int(N.abs().sum()) == 0
    assert bool((lab == 1).all())                      # Regulation 2


def test_disjoint_classes_all_candidates_coherent():
    rng = np.random.default_rng(12)
    XA = igdata.random_words(rng, 70, 64, "half")                 # items 0..63
    XN = np.zeros((75, 2), np.uint64)
    XN[:, 1] = igdata.random_words(rng, 75, 64, "half")[:, 0]     # items 64..127
    XA = np.concatenate([XA, np.zeros((70, 1), np.uint64)], 1)
    rows = np.concatenate([XA, XN])
    labels = np.array([1] * 70 + [0] * 75, np.uint8)
    m = gpu_fit(rows, labels)
    info = m.info()
    assert info["n_patterns"] == info["n_candidates"]
    assert_model_equal(m, oracle.fit(rows, labels))


def test_single_record_classes_and_duplicates():
    rows = np.array([[0b1011], [0b0110]], np.uint64)
    m = gpu_fit(rows, [1, 0])
    assert m.patterns(1)[0].tolist() == [[0b1011]]
    assert m.patterns(0)[0].tolist() == [[0b0110]]
    # All records identical within each class: one candidate, the record.
    rows = np.array([[5]] * 9 + [[6]] * 4, np.uint64)
    m = gpu_fit(rows, [1] * 9 + [0] * 4)
    assert m.patterns(1)[1].tolist() == [9] and m.patterns(0)[1].tolist() == [4]
    # Records whose pairwise intersections are all empty.
    rows = np.array([[1 << i] for i in range(20)], np.uint64)
    labels = [1] * 10 + [0] * 10
    assert_model_equal(gpu_fit(rows, labels), oracle.fit(rows, np.array(labels, np.uint8)))


def test_empty_class_rejected():
    rows = np.array([[1], [2], [3]], np.uint64)
    with pytest.raises(ig.IGError) as e:
        gpu_fit(rows, [1, 1, 1])
    assert e.value.code == -1


def test_bad_label_rejected():
    rows = np.array([[1], [2], [3]], np.uint64)
    with pytest.raises(ig.IGError) as e:
        gpu_fit(rows, [1, 2, 0])
    assert e.value.code == -1


def test_hash_table_growth():
    # ~1.1M distinct, nearly all coherent intersections among 1,500 dense
    # records: the dedup table has to double several times.
    rng = np.random.default_rng(13)
    XA = igdata.random_words(rng, 1500, 256, "three_quarters")
    XN = igdata.random_words(rng, 30, 256, "three_quarters")
    rows = np.concatenate([XA, XN])
    labels = np.array([1] * 1500 + [0] * 30, np.uint8)
    m = gpu_fit(rows, labels)
    om = oracle.fit(rows, labels)
    assert om.n_candidates[1] > 1_000_000
    assert_model_equal(m, om)


# ---- seeded workloads -------------------------------------------------------

def _workload_fit(w, r=None, kernel=0):
    d_codes = dev(w.train_codes)
    rows = ig.ig_encode(d_codes, w.cards)
    m = ig.ig_fit(rows, dev(w.train_labels), r=r, subset_kernel=kernel)
    assert m.info()["subset_kernel"] == {0: 4, 1: 1, 2: 2, 3: 3, 4: 4}[kernel]
    return m, oracle.encode(w.train_codes, w.cards)


@pytest.mark.parametrize("kernel", KERNELS)
def test_tiny_workload_parity(kernel):
    w = igdata.tiny()
    m, rows = _workload_fit(w, kernel=kernel)
    om = oracle.fit(rows, w.train_labels)
    assert_model_equal(m, om)
    assert_scores_equal(m, om, oracle.encode(w.test_codes, w.cards))


@pytest.mark.parametrize("kernel", KERNELS)
def test_tiny_workload_regulation3(kernel):
    w = igdata.tiny()
    m, rows = _workload_fit(w, r=0.568, kernel=kernel)
    om = oracle.fit(rows, w.train_labels, r=0.568)
    mu, sigma, r, thr = m.info()["reg3"]
    assert (mu, sigma, r, thr) == om.reg3          # same fp64 formula and order
    assert_scores_equal(m, om, oracle.encode(w.test_codes, w.cards))


@pytest.fixture(scope="module")
def nsl15k_oracle():
    w = igdata.nsl15k()
    rows = oracle.encode(w.train_codes, w.cards)
    return w, oracle.fit(rows, w.train_labels)


@pytest.fixture(scope="module", params=KERNELS, ids=["lop3", "tcgen05", "index", "index-tc"])
def nsl15k(request, nsl15k_oracle):
    w, om = nsl15k_oracle
    m, _ = _workload_fit(w, kernel=request.param)
    return w, m, om


def test_nsl15k_fit_parity(nsl15k):
    w, m, om = nsl15k
    assert_model_equal(m, om)
    assert sum(m.info()["n_patterns"]) > 100_000


def test_nsl15k_score_parity(nsl15k):
    w, m, om = nsl15k
    assert_scores_equal(m, om, oracle.encode(w.test_codes, w.cards))


def test_evidence_wide_sums_path(nsl15k_oracle, monkeypatch):
    # The tensor-core evidence kernel sums a warp's hits per record in 32-bit
    # shared partial sums when every score is below 2^26 (always true at
    # these shapes), and otherwise adds each hit with its own 64-bit atomic;
    # the test hook forces the second path on the same data.
    w, om = nsl15k_oracle
    m, _ = _workload_fit(w, kernel=4)
    test = oracle.encode(w.test_codes, w.cards)
    assert_scores_equal(m, om, test)
    monkeypatch.setenv("IG_EVIDENCE_WIDE_SUMS", "1")
    assert_scores_equal(m, om, test)


def test_nsl15k_deterministic_and_permutation_invariant(nsl15k):
    w, m, om = nsl15k
    perm = np.random.default_rng(5).permutation(w.train_codes.shape[0])
    rows = ig.ig_encode(dev(w.train_codes[perm]), w.cards)
    m2 = ig.ig_fit(rows, dev(w.train_labels[perm]))
    for cls in (0, 1):
        a, b = m.patterns(cls), m2.patterns(cls)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_host_buffer_path(nsl15k):
    w, m, om = nsl15k
    rows = ig.ig_encode(w.train_codes, w.cards)          # numpy in -> numpy out
    assert isinstance(rows, np.ndarray)
    mh = ig.ig_fit(rows, w.train_labels)
    assert_model_equal(mh, om)
    test = ig.ig_encode(w.test_codes[:3000], w.cards)
    A, N, lab = ig.ig_score(mh, test)
    oA, oN, olab = oracle.score(om, test)
    assert np.array_equal(A, oA) and np.array_equal(N, oN) and np.array_equal(lab, olab)


def test_save_load_roundtrip(nsl15k, tmp_path):
    w, m, om = nsl15k
    path = str(tmp_path / "model.ig")
    m.save(path)
    m2 = ig.ig_model_load(path)
    assert_model_equal(m2, om)
    test = oracle.encode(w.test_codes[:500], w.cards)
    assert_scores_equal(m2, om, test)


def _golden_digests():
    """The oracle's digests of the full-size workloads, and the digest
    function that wrote them (tests/golden/make_digests.py)."""
    return golden_digests.stored(), golden_digests.writer().digest


def _gpu_digest(digest, m, test_rows):
    info = m.info()
    pats = {c: m.patterns(c) for c in (0, 1)}
    A, N, lab = ig.ig_score(m, test_rows)
    return digest(info["n_candidates"], {c: pats[c][0] for c in (0, 1)},
                  {c: pats[c][1] for c in (0, 1)}, {c: pats[c][2] for c in (0, 1)},
                  host(A, np.int64), host(N, np.int64), host(lab, np.uint8)), info


def test_nsl148k_full_parity():
    # Full-size fit and all 133,200 test records' scores against the
    # oracle's digest of the same workload (library default kernel, as the
    # benchmark runs it).
    golden, digest = _golden_digests()
    w = igdata.nsl148k()
    m, _ = _workload_fit(w)
    got, info = _gpu_digest(digest, m, ig.ig_encode(dev(w.test_codes), w.cards))
    want = golden[w.name]
    assert list(info["n_patterns"]) == want["n_patterns"]
    assert list(info["n_candidates"]) == want["n_candidates"]
    assert got == want["sha256"], "148k output differs from the oracle's"


# ---- batched problems -------------------------------------------------------

def test_batched_fit_all_problems_match_single_fits_and_oracle():
    # All 64 problems of the batched workload in one ig_fit_batched call:
    # each model equals its own ig_fit, and each problem's whole output
    # (model and test scores) equals the oracle's digest.
    golden, digest = _golden_digests()
    probs = igdata.batched(igdata.BATCHED_PROBLEMS)
    enc = []
    for w in probs:
        enc.append((ig.ig_encode(dev(w.train_codes), w.cards), dev(w.train_labels)))
    batched = ig.ig_fit_batched(enc)
    widths = set()
    for i, (w, mb) in enumerate(zip(probs, batched)):
        single = ig.ig_fit(*enc[i])
        for cls in (0, 1):
            assert all(np.array_equal(x, y) for x, y in zip(mb.patterns(cls), single.patterns(cls)))
        single.free()
        got, _ = _gpu_digest(digest, mb, ig.ig_encode(dev(w.test_codes), w.cards))
        assert got == golden[w.name]["sha256"], f"problem {i} differs from the oracle"
        widths.add(w.meta["width"])
        mb.free()
    assert len(widths) == 4


def test_batched_pair_stage_with_table_growth(monkeypatch):
    # The batched candidate stage with the usual (small) first tables: the
    # distinct-heavy batched problems overflow them, so tables grow, are
    # rehashed and their bands replayed in further launches.  Every model
    # still equals its problem's oracle digest.
    monkeypatch.setenv("IG_TEST_SMALL_TABLES", "1")
    golden, digest = _golden_digests()
    probs = igdata.batched(igdata.BATCHED_PROBLEMS)[:24]
    enc = [(ig.ig_encode(dev(w.train_codes), w.cards), dev(w.train_labels)) for w in probs]
    launches0 = ig.launch_count()
    ig.prof_enable(True)
    ig.prof_reset()
    try:
        batched = ig.ig_fit_batched(enc)
        torch.cuda.synchronize()
        stages = ig.prof_read()
    finally:
        ig.prof_enable(False)
    assert ig.launch_count() > launches0
    assert stages["rehash"][1] > 0          # some table grew
    for w, mb in zip(probs, batched):
        got, _ = _gpu_digest(digest, mb, ig.ig_encode(dev(w.test_codes), w.cards))
        assert got == golden[w.name]["sha256"], f"{w.name} differs from the oracle"
        mb.free()


def test_batched_pair_stage_is_one_launch():
    # With room for every pair, no table grows: the pair tiles of every
    # class of every problem (all word counts) run in one launch.
    probs = igdata.batched(igdata.BATCHED_PROBLEMS)
    enc = [(ig.ig_encode(dev(w.train_codes), w.cards), dev(w.train_labels)) for w in probs]
    ig.prof_enable(True)
    ig.prof_reset()
    try:
        models = ig.ig_fit_batched(enc)
        torch.cuda.synchronize()
        stages = ig.prof_read()
    finally:
        ig.prof_enable(False)
    assert stages["pair_insert"][1] == 1
    assert stages["rehash"][1] == 0
    assert len({int(r.shape[1]) for r, _ in enc}) == 4
    for m in models:
        m.free()


def _as_np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def test_batched_scoring_matches_single_calls():
    # ig_score_batched over independent (model, rows) jobs -- device and host
    # arrays, jobs sharing a model, an empty batch -- equals one ig_score per
    # job; a failing job is reported by number.
    probs = igdata.batched(igdata.BATCHED_PROBLEMS)[:12]
    enc = [(ig.ig_encode(dev(w.train_codes), w.cards), dev(w.train_labels)) for w in probs]
    models = ig.ig_fit_batched(enc)
    jobs = [(m, ig.ig_encode(dev(w.test_codes), w.cards)) for w, m in zip(probs, models)]
    jobs.append((models[0], jobs[0][1][:0]))                             # empty
    jobs.append((models[1], jobs[1][1].cpu().numpy().view(np.uint64)))   # host arrays
    jobs.append((models[1], jobs[1][1][:17]))                            # shared model
    got = ig.ig_score_batched(jobs, lanes=4)
    for (m, rows), (A, N, lab) in zip(jobs, got):
        rA, rN, rlab = ig.ig_score(m, rows)
        assert np.array_equal(_as_np(A), _as_np(rA))
        assert np.array_equal(_as_np(N), _as_np(rN))
        assert np.array_equal(_as_np(lab), _as_np(rlab))
    assert any(int(_as_np(A).max(initial=0)) > 0 for A, _, _ in got)
    lib = ig.load()
    rows = jobs[0][1]
    bufs = [torch.empty(rows.shape[0], dtype=torch.int64, device=rows.device) for _ in range(4)]
    labs = [torch.empty(rows.shape[0], dtype=torch.uint8, device=rows.device) for _ in range(2)]
    arr = (ig.ig_score_job * 2)()
    arr[0] = ig.ig_score_job(models[0].handle, rows.data_ptr(), rows.shape[0], bufs[0].data_ptr(),
                             bufs[1].data_ptr(), labs[0].data_ptr())
    arr[1] = ig.ig_score_job(None, rows.data_ptr(), rows.shape[0], bufs[2].data_ptr(),
                             bufs[3].data_ptr(), labs[1].data_ptr())
    assert lib.ig_score_batched(arr, 2, 2, None) != 0
    assert b"job 1" in lib.ig_last_error()
    torch.cuda.synchronize()
    for m in models:
        m.free()


def test_batched_fit_reports_failing_problem():
    good = (np.array([[1], [2], [3]], np.uint64), np.array([1, 0, 1], np.uint8))
    bad = (np.array([[1], [2]], np.uint64), np.array([1, 1], np.uint8))   # one class only
    with pytest.raises(ig.IGError, match="problem 1"):
        ig.ig_fit_batched([good, bad, good])
