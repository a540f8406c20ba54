"""Host-side bookkeeping of bench.py (no GPU): the test counts the metric is
built on (Eq. 2, Eq. 3, Eq. 4), the choice of the dominant stage, the
roofline arithmetic, the DRAM-traffic table's workload and hash checks, and
the parsing of the clock and throttle-reason samples."""
import hashlib
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("ig_bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0}


@pytest.fixture
def fixed_peaks(monkeypatch):
    monkeypatch.setattr(bench, "load_peaks", lambda: dict(PEAKS))


def info(**kw):
    base = {"n_train": [10, 20], "n_candidates": [100, 200], "n_patterns": [30, 40],
            "n_pairs": [45, 190], "coherence_tests": [0, 0], "coherence_tests_idx": [0, 0],
            "coherence_tests_tc": [0, 0], "subset_kernel": 4}
    base.update(kw)
    return base


def test_nominal_tests_follow_the_definitions():
    # Eq. 3: every candidate of class c against every record of the other
    # class; Eq. 2: every pattern against its own class; Eq. 4: every test
    # flow against every pattern.  Index 0 = normal, 1 = attack.
    t = bench.nominal_tests(info(), 7)
    assert t["coherence"] == 200 * 10 + 100 * 20
    assert t["support"] == 40 * 20 + 30 * 10
    assert t["evidence"] == 7 * (30 + 40)
    assert t["total"] == t["coherence"] + t["support"] + t["evidence"]


def test_dominant_stage_is_the_largest_single_kernel_stage():
    stages = {"pair_insert": (1.0, 2, 0), "index_build": (9.0, 10, 0),
              "evidence_idx": (2.0, 2, 10), "compact": (0.5, 2, 0)}
    # index_build spans several kernels and never heads the roofline.
    assert bench.dominant_stage(stages) == "evidence_idx"


def test_fused_kernel_roofline_counts_gemm_flops(fixed_peaks):
    # 1e9 executed tests of 2 x 64 x K flops in 2 ms, K = 8.
    r = bench.stage_roofline("evidence_idx", 2.0, 2, 10**9, info(), 8, None, 1)
    assert r["kernel"] == "subset_tc_fused_kernel<8, SUM>"
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(1e9 * 2 * 64 * 8 / 2e-3 / 1e12)
    assert r["peak"] == pytest.approx(2 * PEAKS["bf16_tflops"])
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["avg_launch_ms"] == pytest.approx(1.0)


def test_integer_pipe_roofline_counts_lop3(fixed_peaks):
    r = bench.stage_roofline("evidence_idx", 1.0, 1, 10**9, info(subset_kernel=3), 8,
                             {"sm_max_mhz": 2000.0}, 1)
    assert r["kernel"] == "grouped_subset_kernel<8, SUM>"
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(1e9 * 2 * 8 / 1e-3 / 1e12)
    assert r["peak"] == pytest.approx(bench.LOP3_PER_SM_PER_CLK * 152 * 2000.0 * 1e6 / 1e12)


def test_pair_insert_byte_model(fixed_peaks):
    # Per pair (i < j, plus each record with itself) one stored key of 8K
    # bytes compared; per distinct key one 8K-byte write.
    i = info()
    r = bench.stage_roofline("pair_insert", 1.0, 2, 0, i, 8, None, 3)
    pairs = (45 + 190 + 10 + 20) * 3
    keys = (100 + 200) * 3
    assert r["bound"] == "hbm"
    assert r["algorithmic_bytes_per_launch"] == (pairs + keys) * 64 // 2
    assert r["achieved"] == pytest.approx((pairs + keys) * 64 / 1e-3 / 1e9)
    assert r["peak"] == PEAKS["hbm_gbs"]


def test_pair_insert_l2_accesses(fixed_peaks, monkeypatch):
    # With a probed random-L2 rate: one slot access per pair and one claim
    # per distinct key, against the probed 16-byte loads per second.
    monkeypatch.setattr(bench, "PROBED", {"l2_random": 16.0e12})
    i = info()
    r = bench.stage_roofline("pair_insert", 1.0, 2, 0, i, 8, None, 3)
    pairs = (45 + 190 + 10 + 20) * 3
    keys = (100 + 200) * 3
    assert r["bound"] == "l2"
    assert r["algorithmic_accesses_per_launch"] == (pairs + keys) // 2
    assert r["achieved"] == pytest.approx((pairs + keys) / 1e-3 / 1e9)
    assert r["peak"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)


def test_roofline_head_from_timed_steps_breakdown_from_warmup(fixed_peaks):
    warm = {"pair_insert": (4.0, 4, 0), "evidence_idx": (2.0, 4, 10**9)}
    timed = {"pair_insert": (3.0, 6, 0), "evidence_idx": (0.0, 0, 10**9)}
    head = bench.roofline(timed, info(), 8, None, 3, warm=warm, warm_steps=2)
    assert head["stage"] == "pair_insert"
    assert head["avg_launch_ms"] == pytest.approx(0.5)          # timed: 3 ms / 6 launches
    assert head["all_kernels"]["pair_insert"]["ms_per_step"] == pytest.approx(2.0)   # warm
    assert head["all_kernels"]["evidence_idx"]["ms_per_step"] == pytest.approx(1.0)


def test_traffic_table_entries_are_checked_against_their_sources():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        table = json.load(f)
    for name, rec in table.items():
        if name.startswith("_"):
            continue
        src = os.path.join(ROOT, rec["source"])
        assert os.path.exists(src), name
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for workload, per in rec["by_workload"].items():
            expect = per["bytes_per_launch"] if digest == rec["source_sha256_16"] else None
            assert bench.dram_traffic(name, workload) == expect
        assert bench.dram_traffic(name, "some-other-workload") is None
    assert bench.dram_traffic("no_such_kernel", "ig-nsl-15k-50/50") is None


def test_traffic_lookup_drops_a_changed_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    table = {"k": {"source": "k.cu", "source_sha256_16": digest,
                   "by_workload": {"w": {"bytes_per_launch": 123, "launches_captured": 2}}}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.dram_traffic("k", "w") == 123
    src.write_text("kernel v2\n")
    assert bench.dram_traffic("k", "w") is None


def test_clock_samples_parse_median_max_and_reasons(tmp_path):
    # nvidia-smi rows (csv, no header, no units): index, clocks.sm,
    # clocks.max.sm, power, active reasons, then the four reasons read.
    rows = ["0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1400.2, 0x0000000000000008, Active, Not Active, Not Active, Active",
            "garbage line",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class Done:
        pass
    s = bench.ClockSampler(0)
    s.proc = Done()
    s.tmp = open(path)
    out = s.summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_peaks_fall_back_when_unmeasured(monkeypatch):
    # Without the measured peaks file the rooflines use the stated fallback
    # figures and say so.
    monkeypatch.setattr(bench, "load_peaks", lambda: None)
    r = bench.stage_roofline("evidence_idx", 2.0, 2, 10**9, info(), 8, None, 1)
    assert r["peak"] == pytest.approx(2 * bench.FALLBACK_BF16_TFLOPS)
    assert "fallback" in r["peak_source"]
