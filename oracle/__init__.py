"""CPU oracle for Interpretable Generalization -- TEST INFRASTRUCTURE ONLY.

A plain, slow statement of the IG hot path (paper Section 3.1, Eq. 1-4,
Regulations 1-3; the subset test in the form of Eq. 6), used to check the
CUDA library.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and never imports it.

The arithmetic lives in ``ig_oracle.cpp`` (plain C++ loops, compiled with
g++ on first use); this module only moves numpy arrays in and out and strings
the steps together in the paper's order:

    fit:   split records by class
           -> B^c (Eq. 1) -> keep coherent candidates (Eq. 3 / Eq. 6)
           -> supports f_c and scores S_c = f_c * |b|^2 (Eq. 2)
           -> optional Regulation 3 statistics over the training normals
    score: A(x), N(x) (Eq. 4) -> labels (Regulations 1-3)

Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ig_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libig_oracle.so")
_lib = None

NORMAL = 0
ATTACK = 1


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no SIMD or -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-ffp-contract=off",
           "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "oracle_encode": (ctypes.c_int, [P, I64, I32, P, I32, P]),
        "oracle_candidates": (P, [P, I64, I32]),
        "oracle_list_rows": (I64, [P]),
        "oracle_list_copy": (None, [P, P]),
        "oracle_list_free": (None, [P]),
        "oracle_coherent": (None, [P, I64, P, I64, I32, P, ctypes.c_int]),
        "oracle_support": (None, [P, I64, P, I64, I32, P, P, ctypes.c_int]),
        "oracle_evidence": (None, [P, P, I64, P, I64, I32, P, ctypes.c_int]),
        "oracle_pattern_score": (None, [P, I64, I32, P, P]),
        "oracle_reg3_stats": (None, [P, I64, P, P]),
        "oracle_labels": (None, [P, P, I64, ctypes.c_int, D, P]),
        "oracle_reg3_threshold": (D, [D, D, D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _rows(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.ndim != 2:
        raise ValueError("expected a [rows, K] uint64 array")
    return a


def default_threads() -> int:
    return os.cpu_count() or 1


def encode(codes, cards) -> np.ndarray:
    """Section 3.1 / Eq. 5: one-hot items packed into uint64[n, K]."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    cards = np.ascontiguousarray(cards, dtype=np.uint16)
    n, F = codes.shape
    K = (int(cards.astype(np.int64).sum()) + 63) // 64
    out = np.zeros((n, K), dtype=np.uint64)
    rc = _load().oracle_encode(_ptr(codes), n, F, _ptr(cards), K, _ptr(out))
    if rc != 0:
        raise ValueError("code out of range for its feature")
    return out


def candidates(rows) -> np.ndarray:
    """Eq. 1: B^c in canonical order (ascending, word K-1 most significant)."""
    rows = _rows(rows)
    n, K = rows.shape
    lib = _load()
    h = lib.oracle_candidates(_ptr(rows), n, K)
    try:
        out = np.empty((lib.oracle_list_rows(h), K), dtype=np.uint64)
        if out.size:
            lib.oracle_list_copy(h, _ptr(out))
    finally:
        lib.oracle_list_free(h)
    return out


def coherent(cand, opposite, threads: int | None = None) -> np.ndarray:
    """Eq. 3 / Eq. 6: True where no opposite-class record contains b."""
    cand, opposite = _rows(cand), _rows(opposite)
    K = cand.shape[1]
    assert opposite.shape[1] == K or opposite.shape[0] == 0
    out = np.zeros(cand.shape[0], dtype=np.uint8)
    _load().oracle_coherent(_ptr(cand), cand.shape[0], _ptr(opposite),
                            opposite.shape[0], K, _ptr(out),
                            threads or default_threads())
    return out.astype(bool)


def support(patterns, same, threads: int | None = None):
    """Eq. 2: (f_c(b), S_c(b) = f_c(b) * |b|^2) for every pattern b."""
    patterns, same = _rows(patterns), _rows(same)
    P, K = patterns.shape
    f = np.zeros(P, dtype=np.uint32)
    S = np.zeros(P, dtype=np.uint64)
    _load().oracle_support(_ptr(patterns), P, _ptr(same), same.shape[0], K,
                           _ptr(f), _ptr(S), threads or default_threads())
    return f, S


def pattern_score(patterns, f) -> np.ndarray:
    """Eq. 2 for given supports: S(b) = f(b) * |b|^2 for every pattern b."""
    patterns = _rows(patterns)
    f = np.ascontiguousarray(f, dtype=np.uint32)
    S = np.zeros(patterns.shape[0], dtype=np.uint64)
    _load().oracle_pattern_score(_ptr(patterns), patterns.shape[0], patterns.shape[1],
                                 _ptr(f), _ptr(S))
    return S


def model_from_patterns(patterns: dict, support: dict) -> "Model":
    """A model holding given dictionaries P^- (class 0) and P^+ (class 1)
    with their supports: canonical order (ascending, word K-1 most
    significant) and the scores of Eq. 2."""
    K = None
    pats, sups, scos = {}, {}, {}
    for c in (NORMAL, ATTACK):
        P = _rows(patterns[c])
        K = P.shape[1]
        order = np.lexsort(P.T) if P.shape[0] else np.zeros(0, np.int64)
        pats[c] = np.ascontiguousarray(P[order])
        sups[c] = np.ascontiguousarray(np.asarray(support[c], np.uint32)[order])
        scos[c] = pattern_score(pats[c], sups[c])
    return Model(K, pats, sups, scos, {NORMAL: 0, ATTACK: 0}, None)


def evidence(patterns, S, rows, threads: int | None = None) -> np.ndarray:
    """Eq. 4: sum of S(b) over patterns b contained in each row (int64)."""
    patterns, rows = _rows(patterns), _rows(rows)
    S = np.ascontiguousarray(S, dtype=np.uint64)
    out = np.zeros(rows.shape[0], dtype=np.int64)
    K = rows.shape[1]
    _load().oracle_evidence(_ptr(patterns), _ptr(S), patterns.shape[0],
                            _ptr(rows), rows.shape[0], K, _ptr(out),
                            threads or default_threads())
    return out


def reg3_stats(N) -> tuple[float, float]:
    """Regulation 3: mean and population std of N (fp64, index order)."""
    N = np.ascontiguousarray(N, dtype=np.int64)
    mu, sigma = ctypes.c_double(), ctypes.c_double()
    _load().oracle_reg3_stats(_ptr(N), N.shape[0], ctypes.byref(mu),
                              ctypes.byref(sigma))
    return mu.value, sigma.value


def reg3_threshold(mu: float, sigma: float, r: float) -> float:
    return float(_load().oracle_reg3_threshold(mu, sigma, r))


def labels(A, N, threshold: float | None = None) -> np.ndarray:
    """Regulations 1-3 (Regulation 3 only when a threshold is given)."""
    A = np.ascontiguousarray(A, dtype=np.int64)
    N = np.ascontiguousarray(N, dtype=np.int64)
    out = np.zeros(A.shape[0], dtype=np.uint8)
    _load().oracle_labels(_ptr(A), _ptr(N), A.shape[0],
                          0 if threshold is None else 1,
                          0.0 if threshold is None else float(threshold),
                          _ptr(out))
    return out


@dataclass
class Model:
    """Fitted IG model: coherent dictionaries P^+ (attack), P^- (normal)."""

    K: int
    patterns: dict          # cls -> uint64[|P^c|, K], canonical order
    support: dict           # cls -> uint32[|P^c|]
    score: dict             # cls -> uint64[|P^c|]
    n_candidates: dict      # cls -> |B^c|
    reg3: tuple | None      # (mu_N, sigma_N, r, threshold) or None


def fit(rows, labels_, r: float | None = None, threads: int | None = None) -> Model:
    """IG training: Eq. 1 -> Eq. 3 -> Eq. 2 per class, then Regulation 3.

    labels_: 1 = attack (class +), 0 = normal (class -).  With r given, the
    Regulation 3 statistics are taken over the training normal records scored
    against P^- (Eq. 4).
    """
    rows = _rows(rows)
    lab = np.asarray(labels_, dtype=np.uint8)
    K = rows.shape[1]
    X = {ATTACK: rows[lab == ATTACK], NORMAL: rows[lab == NORMAL]}
    pats, sup, sco, ncand = {}, {}, {}, {}
    for c in (ATTACK, NORMAL):
        B = candidates(X[c])
        keep = coherent(B, X[1 - c], threads)
        P = np.ascontiguousarray(B[keep])
        f, S = support(P, X[c], threads)
        pats[c], sup[c], sco[c], ncand[c] = P, f, S, B.shape[0]
    reg3 = None
    if r is not None:
        n_train = evidence(pats[NORMAL], sco[NORMAL], X[NORMAL], threads)
        mu, sigma = reg3_stats(n_train)
        reg3 = (mu, sigma, float(r), reg3_threshold(mu, sigma, float(r)))
    return Model(K, pats, sup, sco, ncand, reg3)


def score(model: Model, rows, threads: int | None = None):
    """IG inference: (A, N, labels) for each row (Eq. 4, Regulations 1-3)."""
    rows = _rows(rows)
    A = evidence(model.patterns[ATTACK], model.score[ATTACK], rows, threads)
    N = evidence(model.patterns[NORMAL], model.score[NORMAL], rows, threads)
    thr = None if model.reg3 is None else model.reg3[3]
    return A, N, labels(A, N, thr)
