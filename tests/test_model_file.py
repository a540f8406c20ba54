"""ig_model_load on damaged files (CPU: every case here is rejected, or
passes the file checks, before any device work).

The file is a flat little-endian record: magic, version, K, Regulation 3
flag, its statistics, the per-class counts, then per class the words
(8 K bytes), support (4 bytes) and score (8 bytes) of each pattern.  The
pattern counts must account for the rest of the file exactly, so a damaged
header is reported as IG_E_IO instead of driving a huge allocation.
"""
import os
import shutil
import struct

import pytest

import paper_2507_14222_gb300 as ig
from paper_2507_14222_gb300 import buildlib

IG_E_CUDA, IG_E_IO = -3, -7
MAGIC = b"IGGB300\x00"

pytestmark = pytest.mark.skipif(
    not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")),
    reason="nvcc not available")


@pytest.fixture(scope="module", autouse=True)
def lib():
    buildlib.build()
    return ig.load()


def _file(path, K=1, n_pat=(2, 1), data=None, magic=MAGIC, version=1):
    head = magic + struct.pack("<4I", version, K, 0, 0) + struct.pack("<4d", 0, 0, 0, 0)
    head += struct.pack("<8q", 10, 10, 5, 5, 45, 45, *n_pat)
    if data is None:
        data = bytes(sum(max(0, p) for p in n_pat) * (8 * K + 4 + 8))
    with open(path, "wb") as f:
        f.write(head + data)
    return str(path)


def _code(path):
    with pytest.raises(ig.IGError) as e:
        ig.ig_model_load(path)
    return e.value.code


def test_damaged_files_are_rejected(tmp_path):
    assert _code(_file(tmp_path / "huge", n_pat=(1 << 40, 0), data=b"")) == IG_E_IO
    assert _code(_file(tmp_path / "overflow", n_pat=(1 << 62, 1 << 62), data=b"")) == IG_E_IO
    assert _code(_file(tmp_path / "negative", n_pat=(-1, 2))) == IG_E_IO
    assert _code(_file(tmp_path / "short", data=bytes(3 * 20 - 1))) == IG_E_IO
    assert _code(_file(tmp_path / "long", data=bytes(3 * 20 + 1))) == IG_E_IO
    assert _code(_file(tmp_path / "magic", magic=b"NOTIGMOD")) == IG_E_IO
    assert _code(_file(tmp_path / "version", version=99)) == IG_E_IO
    assert _code(_file(tmp_path / "wide", K=17)) == IG_E_IO
    assert _code(str(tmp_path / "absent")) == IG_E_IO


def test_well_formed_file_passes_the_checks(tmp_path):
    # Exactly the layout ig_model_save writes: the file checks pass and the
    # load goes on to the device, which this host does not have.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the round trip is tested on it")
    assert _code(_file(tmp_path / "ok", K=3, n_pat=(2, 1))) == IG_E_CUDA
    assert _code(_file(tmp_path / "empty", K=2, n_pat=(0, 0))) == IG_E_CUDA
