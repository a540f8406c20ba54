"""Planted mistakes in the oracle are caught by its pins.

Each case copies ``oracle/``, ``igdata/`` and the oracle's pin tests into a
scratch directory, plants ONE plausible mistake in the copy of the oracle --
a transposed operand, a dropped term or square, a wrong index, bound or sign,
a strict comparison made loose, the wrong class -- builds that copy and runs
the pins there.  A case passes when at least one pin fails on the mutated
copy.  The control case runs the same harness on an unmodified copy and must
pass every pin, so a failure is the planted mistake's and not the harness's.
The oracle under ``oracle/`` is never modified.  CPU only.
"""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CPP, PY, HELP = "ig_oracle.cpp", "__init__.py", "helpers.py"
PINS = {CPP: "test_oracle_pins.py", PY: "test_oracle_pins.py",
        HELP: "test_oracle_helpers_pins.py"}

# (id, file under oracle/, text that occurs exactly once, its replacement)
MUTANTS = [
    # Eq. 6 containment and |b|
    ("contain-transposed", CPP, "if ((p[k] & r[k]) != p[k]) return false;",
     "if ((p[k] & r[k]) != r[k]) return false;"),
    ("contain-word0-only", CPP, "for (int k = 0; k < K; ++k)\n    if ((p[k] & r[k])",
     "for (int k = 0; k < 1; ++k)\n    if ((p[k] & r[k])"),
    ("size-is-bit-length", CPP, "    w &= w - 1;", "    w >>= 1;"),
    ("size-last-word-dropped", CPP, "for (int k = 0; k < K; ++k) c += items_in_word(b[k]);",
     "for (int k = 0; k + 1 < K; ++k) c += items_in_word(b[k]);"),
    # Eq. 1 candidates, dedup and canonical order
    ("pairs-skip-neighbours", CPP, "for (int64_t j = i + 1; j < n; ++j)",
     "for (int64_t j = i + 2; j < n; ++j)"),
    ("records-not-candidates", CPP, "    push(rows + i * K);\n", ""),
    ("empty-set-kept", CPP, "if (!is_empty(v, K)) all.words", "if (v != nullptr) all.words"),
    ("duplicates-kept", CPP, "if (out->rows() > 0 &&", "if (out->rows() < 0 &&"),
    ("order-word0-major", CPP, "for (int k = K - 1; k >= 0; --k) {\n    if (a[k] != b[k])",
     "for (int k = 0; k < K; ++k) {\n    if (a[k] != b[k])"),
    # Eq. 3 coherence
    ("coherent-inverted", CPP, "out[u] = inside_some ? 0 : 1;", "out[u] = inside_some ? 1 : 0;"),
    ("coherent-skips-first-record", CPP, "for (int64_t t = 0; t < n_opp && !inside_some; ++t)",
     "for (int64_t t = 1; t < n_opp && !inside_some; ++t)"),
    # Eq. 2 supports and scores
    ("score-not-squared", CPP, "S[p] = uint64_t(count) * size * size;",
     "S[p] = uint64_t(count) * size;"),
    ("support-counts-misses", CPP, "if (contained_in(pat + p * K, same + t * K, K)) ++count;",
     "if (!contained_in(pat + p * K, same + t * K, K)) ++count;"),
    ("given-score-cubed", CPP, "S[p] = uint64_t(f[p]) * size * size;",
     "S[p] = uint64_t(f[p]) * size * size * size;"),
    # Eq. 4 evidence
    ("evidence-transposed", CPP, "if (contained_in(pat + p * K, rows + t * K, K)) sum +=",
     "if (contained_in(rows + t * K, pat + p * K, K)) sum +="),
    ("evidence-counts-patterns", CPP, "sum += int64_t(S[p]);", "sum += 1;"),
    ("evidence-32-bit-sum", CPP, "      int64_t sum = 0;", "      int32_t sum = 0;"),
    ("threads-drop-last-row", CPP, "int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);",
     "int64_t lo = t * chunk, hi = std::min<int64_t>(n - 1, lo + chunk);"),
    # Regulations 1-3
    ("reg1-strict", CPP, "(A[t] >= N[t]) ? 1 : 0", "(A[t] > N[t]) ? 1 : 0"),
    # (Dropping Regulation 2 outright changes nothing: A == N == 0 already
    # gives A >= N, attack, under Regulation 1.)
    ("reg2-or-for-and", CPP, "if (A[t] == 0 && N[t] == 0) label = 1;",
     "if (A[t] == 0 || N[t] == 0) label = 1;"),
    ("reg3-loose", CPP, "double(N[t]) < threshold", "double(N[t]) <= threshold"),
    ("reg3-sample-std", CPP, "*sigma = std::sqrt(ss / double(n));",
     "*sigma = std::sqrt(ss / double(n > 1 ? n - 1 : 1));"),
    ("reg3-threshold-sign", CPP, "return mu - scaled;", "return mu + scaled;"),
    ("reg3-mean-over-n-plus-1", CPP, "double mean = sum / double(n);",
     "double mean = sum / double(n + 1);"),
    # Section 3.1 / Eq. 5 encoding
    ("encode-missing-keeps-offset", CPP, "        offset += cards[f];\n        continue;",
     "        continue;"),
    ("encode-range-off-by-one", CPP, "if (v >= cards[f]) return -1;",
     "if (v > cards[f]) return -1;"),
    ("encode-msb-first", CPP, "|= uint64_t(1) << (item % 64);", "|= uint64_t(1) << (63 - item % 64);"),
    # the fit and score steps strung together
    ("fit-coherence-same-class", PY, "keep = coherent(B, X[1 - c], threads)",
     "keep = coherent(B, X[c], threads)"),
    ("fit-support-other-class", PY, "f, S = support(P, X[c], threads)",
     "f, S = support(P, X[1 - c], threads)"),
    ("fit-counts-kept-candidates", PY, "= P, f, S, B.shape[0]", "= P, f, S, P.shape[0]"),
    ("score-classes-swapped", PY,
     "A = evidence(model.patterns[ATTACK], model.score[ATTACK], rows, threads)\n"
     "    N = evidence(model.patterns[NORMAL], model.score[NORMAL], rows, threads)",
     "A = evidence(model.patterns[NORMAL], model.score[NORMAL], rows, threads)\n"
     "    N = evidence(model.patterns[ATTACK], model.score[ATTACK], rows, threads)"),
    ("reg3-stats-over-attacks", PY, "evidence(pats[NORMAL], sco[NORMAL], X[NORMAL], threads)",
     "evidence(pats[NORMAL], sco[NORMAL], X[ATTACK], threads)"),
    ("given-order-word0-major", PY, "order = np.lexsort(P.T) if", "order = np.lexsort(P.T[::-1]) if"),
    ("score-ignores-reg3", PY, "thr = None if model.reg3 is None else model.reg3[3]", "thr = None"),
    ("given-supports-not-reordered", PY,
     "sups[c] = np.ascontiguousarray(np.asarray(support[c], np.uint32)[order])",
     "sups[c] = np.ascontiguousarray(np.asarray(support[c], np.uint32))"),
    # host helpers: discretiser, contradiction filter, metrics, sweep
    ("stats-sample-std", HELP, "return mu, math.sqrt(ss / float(count))",
     "return mu, math.sqrt(ss / float(max(count - 1, 1)))"),
    ("token-truncates", HELP, "return int(np.rint(zs))", "return int(zs)"),
    ("vocab-descending", HELP, "enumerate(sorted(vocab))", "enumerate(sorted(vocab, reverse=True))"),
    ("filter-drops-last-attacks", HELP, "dropped = normal[:k] + attack[:k]",
     "dropped = normal[:k] + attack[len(attack) - k:]"),
    ("filter-mode1-any-class", HELP, "if normal and attack else []", "if normal or attack else []"),
    ("filter-pairs-by-max", HELP, "k = min(len(normal), len(attack))",
     "k = max(len(normal), len(attack))"),
    ("unseen-token-coded-0", HELP, "if t is not None and t in rank:\n                codes[i, f] = rank[t]",
     "if t is not None:\n                codes[i, f] = rank.get(t, 0)"),
    ("constant-column-token-1", HELP, "    if not sigma > 0.0:\n        return 0",
     "    if not sigma > 0.0:\n        return 1"),
    ("decimals-off-by-one", HELP, "scale = float(10 ** int(p))", "scale = float(10 ** (int(p) + 1))"),
    ("precision-uses-fn", HELP, '"precision": _ratio(tp, tp + fp)', '"precision": _ratio(tp, tp + fn)'),
    ("f1-halved", HELP, '"f1": _ratio(2 * tp, 2 * tp + fp + fn)', '"f1": _ratio(tp, tp + fp + fn)'),
    ("auc-ties-dropped", HELP, "two_u += 2 * below + (upto - below)", "two_u += 2 * below"),
    ("auc-score-reversed", HELP, "s = [int(a) - int(n) for a, n in zip(A, N)]",
     "s = [int(n) - int(a) for a, n in zip(A, N)]"),
    ("sweep-loose", HELP, "or float(int(n)) < thr)", "or float(int(n)) <= thr)"),
    ("sweep-threshold-sign", HELP, "thr = mu - (float(r) * sigma)", "thr = mu + (float(r) * sigma)"),
]

_IGNORE = shutil.ignore_patterns("_build", "__pycache__")


def _copy_tree(dst):
    """oracle/, igdata/ and the pin tests (with what they read) under dst."""
    for pkg in ("oracle", "igdata"):
        shutil.copytree(os.path.join(ROOT, pkg), os.path.join(dst, pkg), ignore=_IGNORE)
    tests = os.path.join(dst, "tests")
    os.makedirs(tests)
    for name in ("__init__.py", "conftest.py", "brute.py", *set(PINS.values())):
        shutil.copy2(os.path.join(ROOT, "tests", name), tests)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tests, "golden"),
                    ignore=_IGNORE)


def _build_oracle(dst):
    """Compiles the copy's C++ with the flags the oracle uses for itself."""
    build = os.path.join(dst, "oracle", "_build")
    os.makedirs(build, exist_ok=True)
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-ffp-contract=off", "-shared",
                    "-fPIC", os.path.join(dst, "oracle", CPP), "-o",
                    os.path.join(build, "libig_oracle.so")], check=True)


def _run_pins(dst, pin_file):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", pin_file)],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


@pytest.mark.parametrize("pin_file", sorted(set(PINS.values())))
def test_control_copy_passes_every_pin(tmp_path, pin_file):
    _copy_tree(str(tmp_path))
    _build_oracle(str(tmp_path))
    rc, out = _run_pins(str(tmp_path), pin_file)
    assert rc == 0, out[-3000:]


def _run_mutant(dst, fname, old, new):
    """Plants one mistake in a fresh copy under dst, builds it and runs its pins."""
    _copy_tree(dst)
    path = os.path.join(dst, "oracle", fname)
    with open(path) as f:
        src = f.read()
    if src.count(old) != 1:
        return None, "the text to replace must occur exactly once"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    _build_oracle(dst)
    return _run_pins(dst, PINS[fname])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant's (return code, output), the copies built and pinned
    concurrently (each is an independent scratch tree and process)."""
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        futs = {m[0]: ex.submit(_run_mutant, str(tmp_path_factory.mktemp(m[0])), *m[1:])
                for m in MUTANTS}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, out = outcomes[name]
    assert rc is not None, f"{name}: {out}"
    caught = re.findall(r"^FAILED (\S+)", out, re.M)
    assert rc == 1 and caught, f"{name} was not caught by any pin (rc {rc}):\n{out[-3000:]}"
