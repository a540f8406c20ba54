"""The Python binding rejects arrays the library would misread, before any
library call: tensors of another element size (the library reads 8-byte
words, 2-byte codes, 1-byte labels, 4-byte supports), vectors of the wrong
length, and a cards list that does not match the codes.  CPU only: every case
raises in the binding, so no device work is asked for.
"""
import os
import shutil

import numpy as np
import pytest

import paper_2507_14222_gb300 as ig
from paper_2507_14222_gb300 import buildlib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.skipif(
    not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")),
    reason="nvcc not available")


@pytest.fixture(scope="module", autouse=True)
def lib():
    buildlib.build()
    return ig.load()


def _launches():
    return ig.launch_count()


def test_encode_checks():
    before = _launches()
    with pytest.raises(ValueError, match="16-bit codes"):
        ig.ig_encode(torch.zeros((4, 2), dtype=torch.int32), [3, 5])
    with pytest.raises(ValueError, match="cards"):
        ig.ig_encode(np.zeros((4, 3), np.uint16), [3, 5])
    with pytest.raises(ValueError, match=r"\[n, F\]"):
        ig.ig_encode(np.zeros(4, np.uint16), [3])
    assert _launches() == before


def test_fit_checks():
    before = _launches()
    rows = torch.zeros((10, 2), dtype=torch.int64)
    with pytest.raises(ValueError, match="64-bit words"):
        ig.ig_fit(rows.to(torch.int32), torch.zeros(10, dtype=torch.uint8))
    with pytest.raises(ValueError, match=r"shape \[10\]"):
        ig.ig_fit(rows, torch.zeros(9, dtype=torch.uint8))
    with pytest.raises(ValueError, match="element type"):
        ig.ig_fit(rows, torch.zeros(10, dtype=torch.int64))
    with pytest.raises(ValueError, match=r"shape \[10\]"):
        ig.ig_fit(np.zeros((10, 2), np.uint64), np.zeros((10, 1), np.uint8))
    with pytest.raises(ValueError, match=r"\[n, K\]"):
        ig.ig_fit(np.zeros(10, np.uint64), np.zeros(10, np.uint8))
    assert _launches() == before


def test_fit_batched_names_the_bad_problem():
    good = (np.array([[1], [2], [3]], np.uint64), np.array([1, 0, 1], np.uint8))
    bad = (np.array([[1], [2], [3]], np.uint64), np.array([1, 0], np.uint8))
    with pytest.raises(ValueError, match="problem 1: labels"):
        ig.ig_fit_batched([good, bad, good])
    bad_rows = (torch.zeros((3, 1), dtype=torch.int32), torch.zeros(3, dtype=torch.uint8))
    with pytest.raises(ValueError, match="problem 2: rows"):
        ig.ig_fit_batched([good, good, bad_rows])


def test_model_from_patterns_checks():
    w = np.array([[1, 0], [2, 0]], np.uint64)
    f = np.ones(2, np.uint32)
    with pytest.raises(ValueError, match="same K"):
        ig.ig_model_from_patterns(w, f, w[:, :1].copy(), f)
    with pytest.raises(ValueError, match="class 1: support"):
        ig.ig_model_from_patterns(w, f, w, f[:1].copy())
    with pytest.raises(ValueError, match="class 0: words"):
        ig.ig_model_from_patterns(torch.zeros((2, 2), dtype=torch.int32),
                                  torch.ones(2, dtype=torch.int32), w, f)
    with pytest.raises(ValueError, match="element type"):
        ig.ig_model_from_patterns(w, torch.ones(2, dtype=torch.int64), w, f)


def test_valid_arrays_reach_the_library():
    # The checks pass well-formed arrays through: without a GPU the library
    # itself then fails loudly.
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ig.IGError) as e:
        ig.ig_fit(np.zeros((10, 2), np.uint64), np.zeros(10, np.uint8))
    assert e.value.code == -3
    with pytest.raises(ig.IGError) as e:
        ig.ig_encode(np.zeros((4, 2), np.uint16), [3, 5])
    assert e.value.code == -3
