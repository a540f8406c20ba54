"""bench.py --impl reference: the CPU oracle timed on the host's cores.

It needs no GPU, so the CPU suite runs it as the benchmark does: one JSON line on
rank 0 with the benchmark's metric, unit and workload, a cpu_baseline that
describes the run, and an e2e with no copies; any other rank exits 0 without
work or output.  The benchmark's own arm, on a host without a GPU, exits
non-zero without a result line.
"""
import importlib.util
import json
import os
import subprocess
import sys

import igdata

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("ig_bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout, p.stderr


def test_reference_arm_prints_one_line_on_the_default_workload():
    rc, out, err = _run(None, "--steps", "3", "--warmup", "3")
    assert rc == 0, err[-2000:]
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 3, 3)
    assert d["config"]["workload"] == igdata.nsl148k().name
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] == (os.cpu_count() or 1) and cb["sample"] == d["config"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    rc, out, err = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"},
                        "--steps", "3", "--warmup", "3")
    assert rc == 0, err[-2000:]
    assert out.strip() == ""


def test_own_arm_without_a_gpu_fails_loudly():
    # No CPU fallback: without a CUDA device the benchmark exits non-zero and
    # prints no result line.
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    p = subprocess.run([sys.executable, "bench.py", "--steps", "3", "--warmup", "3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode != 0
    assert not [l for l in p.stdout.splitlines() if l.lstrip().startswith("{")]


def _line(out):
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_arm_batched_and_served_workloads():
    rc, out, err = _run(None, "--workload", "batched", "--steps", "3", "--warmup", "3")
    assert rc == 0, err[-2000:]
    d = _line(out)
    assert d["unit"] == bench.UNIT and d["config"]["workload"] == "ig-batched-64-problems"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    rc, out, err = _run(None, "--workload", "served", "--served-patterns", "3000",
                        "--served-flows", "5000", "--steps", "3", "--warmup", "3")
    assert rc == 0, err[-2000:]
    d = _line(out)
    assert d["unit"] == "flows/s" and d["value"] > 0
    assert d["config"]["workload"] == "ig-served-3000x2-patterns-5000-flows"
    assert d["e2e"]["unit"] == "flows/s"
