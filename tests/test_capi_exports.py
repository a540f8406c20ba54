"""The C ABI library builds, loads and exports every symbol of include/*.h.

No compute happens here: on a machine without a GPU the only calls made are
pure host functions, plus one compute call that must fail loudly (there is no
CPU fallback).
"""
import ctypes
import glob
import os
import re
import shutil

import numpy as np
import pytest

import paper_2507_14222_gb300 as ig
from paper_2507_14222_gb300 import buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ig_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


needs_nvcc = pytest.mark.skipif(
    not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")),
    reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    buildlib.build()
    return ig.load()


@needs_nvcc
def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"ig_encode", "ig_fit", "ig_score", "ig_model_free"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
        assert name in ig.SIGNATURES, f"{name} has no binding signature"


@needs_nvcc
def test_host_only_calls(lib):
    assert lib.ig_prof_stage_name(0) == b"encode"
    assert lib.ig_prof_stage_name(99) == b""
    assert isinstance(lib.ig_last_error(), bytes)


@needs_nvcc
def test_bad_arguments_rejected_before_any_device_work(lib):
    out = ctypes.c_void_p()
    rc = lib.ig_fit(None, None, 0, 8, None, ctypes.byref(out), None)
    assert rc == -1 and out.value is None
    rc = lib.ig_fit(ctypes.c_void_p(1), ctypes.c_void_p(1), 10, 17, None,
                    ctypes.byref(out), None)
    assert rc == -1 and b"K" in lib.ig_last_error()


@needs_nvcc
def test_compute_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    codes = np.zeros((4, 2), np.uint16)
    with pytest.raises(ig.IGError) as e:
        ig.ig_encode(codes, [3, 5])
    assert e.value.code == -3          # IG_E_CUDA: no silent CPU path


def test_missing_library_raises(tmp_path):
    saved = ig._lib
    try:
        ig._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            ig.load(str(tmp_path / "absent.so"))
    finally:
        ig._lib = saved
