"""The stored oracle digests and the function that wrote them
(tests/golden/make_digests.py), for the tests that compare whole outputs."""
import importlib.util
import json
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def writer():
    """tests/golden/make_digests.py as a module."""
    spec = importlib.util.spec_from_file_location("make_digests",
                                                  os.path.join(HERE, "make_digests.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def stored() -> dict:
    """Workload name -> stored entry (sha256, sizes)."""
    with open(os.path.join(HERE, "oracle_digests.json")) as f:
        return json.load(f)["workloads"]
