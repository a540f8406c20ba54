"""The stored oracle digests (tests/golden/oracle_digests.json) still describe
the oracle as it stands.

The GPU tests compare the library's full-size output with these digests, so
a digest that no longer matches the oracle would fail them for the wrong
reason, or let a wrong result pass.  This CPU test recomputes, from the
oracle alone, the digest of every batched problem with at most 1,500
training records (about half of the 64) and checks it, together with the
recorded sizes, against the stored file.
"""
import pytest

import igdata
from tests.golden_digests import stored as _stored, writer as _make_digests


def test_every_workload_has_a_digest():
    stored = _stored()
    names = {igdata.batched_problem(i).name for i in range(igdata.BATCHED_PROBLEMS)}
    names.add(igdata.nsl148k().name)
    names.add("ig-served-1000000x2-patterns-1000000-flows")   # igdata.served() at its defaults
    assert names <= set(stored)
    for entry in stored.values():
        assert len(entry["sha256"]) == 64 and int(entry["sha256"], 16) >= 0


SMALL = [i for i in range(igdata.BATCHED_PROBLEMS)
         if igdata.batched_problem(i).train_codes.shape[0] <= 1500]


@pytest.mark.parametrize("i", SMALL)
def test_batched_digest_reproduces(i):
    md = _make_digests()
    w = igdata.batched_problem(i)
    got = md.oracle_entry(w)
    want = _stored()[w.name]
    for key in ("train", "test", "n_candidates", "n_patterns", "sha256"):
        assert got[key] == want[key], key
