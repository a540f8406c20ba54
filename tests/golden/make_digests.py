"""Writes tests/golden/oracle_digests.json: SHA-256 digests of the CPU
oracle's complete output on the full-size seeded workloads, so that the GPU
tests compare the library's whole output with the oracle's without running
the oracle on the GPU host:

  * ig-nsl-148k-10/90 (14,800 training records; all 133,200 test records
    scored);
  * every one of the 64 batched problems (each fitted on its own, its test
    records scored);
  * the served workload: 1M + 1M given patterns (a model built from them,
    canonical order and Eq. 2 scores) and all 10^6 flows scored (about half
    an hour on 8 cores; run with the argument "served").

Per problem the digest covers, for class 0 (normal) then 1 (attack), the
number of candidates |B^c| (Eq. 1) as a little-endian uint64, then the
canonical pattern words (uint64), supports f_c (uint32) and scores S_c
(uint64) of Eq. 2, then A, N (int64) and the labels (uint8) of Eq. 4 and
Regulations 1-2 over the test records.  Integer results only (Regulation 3
off), so the digests do not depend on the host.

Test infrastructure: calls only oracle/ and the input generator igdata.
Run: python tests/golden/make_digests.py  (several minutes on 8 cores).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import igdata  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_digests.json")


def digest(n_candidates, patterns, support, score, A, N, labels) -> str:
    """The digest the GPU tests recompute from the library's output."""
    h = hashlib.sha256()
    for c in (0, 1):
        h.update(np.asarray([n_candidates[c]], "<u8").tobytes())
        h.update(np.ascontiguousarray(patterns[c], "<u8").tobytes())
        h.update(np.ascontiguousarray(support[c], "<u4").tobytes())
        h.update(np.ascontiguousarray(score[c], "<u8").tobytes())
    h.update(np.ascontiguousarray(A, "<i8").tobytes())
    h.update(np.ascontiguousarray(N, "<i8").tobytes())
    h.update(np.ascontiguousarray(labels, "u1").tobytes())
    return h.hexdigest()


def oracle_entry(w) -> dict:
    rows = oracle.encode(w.train_codes, w.cards)
    test = oracle.encode(w.test_codes, w.cards)
    t0 = time.time()
    m = oracle.fit(rows, w.train_labels)
    A, N, lab = oracle.score(m, test)
    return {"sha256": digest(m.n_candidates, m.patterns, m.support, m.score, A, N, lab),
            "n_candidates": [int(m.n_candidates[0]), int(m.n_candidates[1])],
            "n_patterns": [int(m.patterns[0].shape[0]), int(m.patterns[1].shape[0])],
            "train": int(w.train_codes.shape[0]), "test": int(w.test_codes.shape[0]),
            "oracle_s": round(time.time() - t0, 1)}


def served_entry(sw) -> dict:
    """A model from given patterns has no candidate stage: |B^c| = 0."""
    t0 = time.time()
    m = oracle.model_from_patterns({c: oracle.encode(sw.patterns[c], sw.cards) for c in (0, 1)},
                                   sw.support)
    A, N, lab = oracle.score(m, oracle.encode(sw.flow_codes, sw.cards))
    return {"sha256": digest(m.n_candidates, m.patterns, m.support, m.score, A, N, lab),
            "n_candidates": [int(m.n_candidates[0]), int(m.n_candidates[1])],
            "n_patterns": [int(m.patterns[0].shape[0]), int(m.patterns[1].shape[0])],
            "flows": int(sw.flow_codes.shape[0]),
            "oracle_s": round(time.time() - t0, 1)}


def main():
    out = {"about": "SHA-256 of the CPU oracle's output per workload; written by "
                    "tests/golden/make_digests.py (see its docstring for the byte layout)",
           "workloads": {}}
    which = sys.argv[1:] or ["nsl148k", "batched"]
    if os.path.exists(OUT):
        out = json.load(open(OUT))
    if "nsl148k" in which:
        w = igdata.nsl148k()
        out["workloads"][w.name] = oracle_entry(w)
        print(w.name, out["workloads"][w.name], flush=True)
    if "batched" in which:
        for i in range(igdata.BATCHED_PROBLEMS):
            w = igdata.batched_problem(i)
            out["workloads"][w.name] = oracle_entry(w)
            print(w.name, out["workloads"][w.name], flush=True)
            json.dump(out, open(OUT, "w"), indent=1)
    if "served" in which:
        sw = igdata.served()
        out["workloads"][sw.name] = served_entry(sw)
        print(sw.name, out["workloads"][sw.name], flush=True)
    json.dump(out, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
