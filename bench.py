"""IG hot-path benchmark on synthetic NSL-KDD-shaped data (one JSON line).

A step is one pass of the whole hot path over one workload: encode the
training and test records (Eq. 5), fit (Eq. 1 -> Eq. 3 -> Eq. 2: pairwise
intersections, dedup, coherence, canonical order, supports and scores) and
score the test records (Eq. 4, Regulations 1-3).  Inputs (the discretised
codes and labels) are resident on the device when the timed region starts;
L2 is flushed (a 512 MiB write) before every timed step and each step is
timed with CUDA events on the launching stream.

value = subset tests per second, where the tests of one step are those the
definitions require: |B^c| x n_(other class) for coherence (Eq. 3),
|P^c| x n_c for supports (Eq. 2) and m_test x (|P+| + |P-|) for the
evidence (Eq. 4), summed over both classes.

Also reported: fit wall time, scored flows/s, an end-to-end figure through
the C ABI with host buffers, the roofline of the dominant kernel, the CPU
oracle timed on this host's cores, SM clocks sampled during the timed region
and the number of kernels launched.

--impl reference times the CPU oracle (the only other implementation of the
method here) on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank fits its own independent problem of the same
shape (seed offset by rank); there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import igdata  # noqa: E402

METRIC = "IG fit wall-s & subset tests/s (G/s) vs roofline; scored flows/s, p99 ms"
UNIT = "G subset-tests/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# Integer-pipe peak of the subset test: LOP3 instructions per SM per clock
# (4 sub-partitions x 16 lanes) x 152 SMs x the maximum SM clock.  The
# library's LOP3 probe (ig_probe, run at the start of every bench) measured
# 2.01e13 per second on GB300, the same figure at 2,070 MHz.
LOP3_PER_SM_PER_CLK = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nsl148k",
                    choices=sorted(igdata.WORKLOADS) + ["batched", "served"])
    ap.add_argument("--served-patterns", type=int, default=1_000_000,
                    help="patterns per class of the served workload")
    ap.add_argument("--served-flows", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the batched and served comparisons of the default line")
    ap.add_argument("--kernel", type=int, default=0,
                    help="subset-test form: 0 default, 1 integer pipe, 2 tensor cores, "
                         "3 item index, 4 item index on the tensor cores")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def nominal_tests(info: dict, m_test: int) -> dict:
    """Subset tests the definitions require for one fit + score."""
    nt, U, P = info["n_train"], info["n_candidates"], info["n_patterns"]
    coh = U[1] * nt[0] + U[0] * nt[1]
    sup = P[1] * nt[1] + P[0] * nt[0]
    ev = m_test * (P[0] + P[1])
    return {"coherence": coh, "support": sup, "evidence": ev,
            "total": coh + sup + ev}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.tmp:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.tmp.flush()
        rows = list(csv.reader(io.StringIO(open(self.tmp.name).read())))
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import torch

    import paper_2507_14222_gb300 as ig

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ig.build()
    ig.load()
    probes = run_probes(ig)
    if args.workload == "batched":
        return run_batched(args, ig, torch, rank, world, local)
    if args.workload == "served":
        return run_served(args, ig, torch, rank, world, local)

    from paper_2507_14222_gb300 import replicas
    w = {"tiny": lambda: igdata.tiny(replicas.replica_seed(1001, rank)),
         "nsl15k": lambda: igdata.nsl15k(replicas.replica_seed(1002, rank)),
         "nsl148k": lambda: igdata.nsl148k(replicas.replica_seed(1003, rank))}[args.workload]()
    cards = w.cards
    d_tr = torch.from_numpy(w.train_codes.view(np.int16)).cuda()
    d_lab = torch.from_numpy(w.train_labels).cuda()
    d_te = torch.from_numpy(w.test_codes.view(np.int16)).cuda()
    m_test = w.test_codes.shape[0]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        rows = ig.ig_encode(d_tr, cards)
        test_rows = ig.ig_encode(d_te, cards)
        model = ig.ig_fit(rows, d_lab, subset_kernel=args.kernel)
        out = ig.ig_score(model, test_rows)
        return model, out

    # Warm-up steps after the first carry events around every stage (the
    # per-stage breakdown); in the timed steps only the dominant kernel's
    # stage does, so that the others run without event overhead.
    info = None
    first_profiled = min(1, args.warmup - 1)
    for i in range(args.warmup):
        if i == first_profiled:
            ig.prof_select(None)
            ig.prof_reset()
            ig.prof_enable(True)
        model, _out = step()
        info = model.info()
        model.free()
    torch.cuda.synchronize()
    ig.prof_enable(False)
    warm = ig.prof_read()
    n_warm = args.warmup - first_profiled
    tests = nominal_tests(info, m_test)
    top = dominant_stage(warm)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fit_ms = []
    ig.prof_select([top])
    ig.prof_reset()
    ig.prof_enable(True)
    launches0 = ig.launch_count()
    replicas.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            rows = ig.ig_encode(d_tr, cards)
            test_rows = ig.ig_encode(d_te, cards)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            model = ig.ig_fit(rows, d_lab, subset_kernel=args.kernel)
            f1.record(stream)
            ig.ig_score(model, test_rows)
            ends[i].record(stream)
            model.free()
            torch.cuda.synchronize()
            fit_ms.append(f0.elapsed_time(f1))
        torch.cuda.synchronize()
    replicas.barrier()
    launches = ig.launch_count() - launches0
    ig.prof_enable(False)
    stages = ig.prof_read()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # Slowest rank's time; every rank's own tests (their problems differ).
    total_ms, job_tests = replicas.job_totals(sum(step_ms), tests["total"] * args.steps,
                                              device="cuda")
    ms_per_step = total_ms / args.steps
    value = job_tests / args.steps / (ms_per_step * 1e-3) / 1e9

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    executed = {
        "coherence": sum(info["coherence_tests"]),
        "support": sum(info["support_tests"]),
        "evidence": sum(stages.get(k, (0, 0, 0))[2] for k in
                        ("evidence_idx", "evidence_tc", "evidence")) // max(1, args.steps)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": w.name, "train_records": int(w.train_codes.shape[0]),
                   "test_records": int(m_test), "features": w.n_features,
                   "items_L": w.n_items, "words_K": w.n_words,
                   "l2": "flushed before every timed step (512 MiB write)",
                   "parallelism": f"{world} independent problems" if world > 1 else "single"},
        "fit_s": statistics.median(fit_ms) * 1e-3,
        "flows_per_s": m_test / (ms_per_step * 1e-3),
        "tests_per_step": tests,
        "patterns": {"attack": info["n_patterns"][1], "normal": info["n_patterns"][0],
                     "candidates": list(info["n_candidates"][::-1])},
        "subset_kernel": {1: "lop3", 2: "tcgen05", 3: "item-index",
                          4: "item-index-tcgen05"}[info["subset_kernel"]],
        "executed_tests_per_step": executed,
        # The same step's rate counted in executed subset tests (after the
        # item index's exact pruning and the coherence windows' early drops)
        # instead of the tests the definitions require.
        "executed_value": sum(executed.values()) / (ms_per_step * 1e-3) / 1e9,
        "stages_ms_per_step": {k: round(v[0] / n_warm, 4) for k, v in warm.items() if v[1]},
        "stage_timing": f"stages: {n_warm} profiled warm-up step(s); timed steps: events "
                        f"around the {top} stage only",
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "probes": {k: (round(v / 1e12, 2) if isinstance(v, float) else v)
                   for k, v in probes.items()},
        "probes_unit": "1e12 per second (LOP3 instructions, bytes of L2 loads, MMA flops)",
    }
    kt = 1
    while kt < w.n_words:
        kt *= 2
    line["roofline"] = roofline(stages, info, kt, line["clocks"], args.steps, w.name,
                                warm=warm, warm_steps=n_warm)
    if not args.no_e2e:
        line["e2e"] = e2e_host_buffers(ig, w, tests, max(2, min(args.steps, 5)))
    if not args.no_extras and world == 1:
        # The batched and served forms against their plain counterparts, on
        # the same GPU in the same run (config 4 and config 5 shapes).
        line["batched"] = measure_batched(args, ig, torch, local, 3, 1)
        line["served"] = measure_served(args, ig, torch, local)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_batched(args, ig, torch, local, steps, warmup, seed=2000):
    """64 independent problems per step, each fitted and its test records
    scored: one ig_fit_batched and one ig_score_batched call against one
    ig_fit and one ig_score per problem (the plain per-problem launches),
    same inputs, same process.  Models and scores must be identical.
    Returns the measurements (ms per step of each form)."""
    probs = igdata.batched(igdata.BATCHED_PROBLEMS, seed)
    dev = []
    for w in probs:
        dev.append((torch.from_numpy(w.train_codes.view(np.int16)).cuda(),
                    torch.from_numpy(w.train_labels).cuda(),
                    torch.from_numpy(w.test_codes.view(np.int16)).cuda(), w.cards))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def encode_all():
        return [(ig.ig_encode(c, cards), lab, ig.ig_encode(t, cards)) for c, lab, t, cards in dev]

    # Tiling and subset-test form per (K, size) group, tuned once per GPU
    # (cached), outside the timed region; both forms use the same choices.
    from paper_2507_14222_gb300 import autotune
    tuner = autotune.Autotuner()
    enc0 = encode_all()
    tuned = tuner.tune(enc0) if args.kernel == 0 else {}
    per_params = [tuner.params_for(int(r.shape[1]), int(r.shape[0])) if args.kernel == 0
                  else None for r, _, _ in enc0]
    del enc0

    def step(batched):
        enc = encode_all()
        if batched:
            # One lane: the candidate stage of all problems is one launch either
            # way, and on this GPU-bound mix more lanes measured no faster once
            # warm (the first multi-lane call is, later ones not).
            models = ig.ig_fit_batched([(r, lab) for r, lab, _ in enc],
                                       subset_kernel=args.kernel,
                                       per_problem_params=per_params, lanes=1)
            scores = ig.ig_score_batched([(mdl, te) for mdl, (_, _, te) in zip(models, enc)],
                                         lanes=1)
            return models, scores
        else:
            models = []
            for (r, lab, _), pp in zip(enc, per_params):
                if pp is None:
                    models.append(ig.ig_fit(r, lab, subset_kernel=args.kernel))
                else:
                    models.append(ig.ig_fit(r, lab, subset_kernel=pp.subset_kernel,
                                            index_max_q=pp.index_max_q,
                                            index_flip_factor=pp.index_flip_factor))
        scores = [ig.ig_score(mdl, te) for mdl, (_, _, te) in zip(models, enc)]
        return models, scores

    def timed(batched, n):
        ms, last = [], None
        for _ in range(n):
            if last:
                for mdl in last:
                    mdl.free()
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            models, scores = step(batched)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            last = models
        return ms, last, scores

    for _ in range(warmup):
        for form in (True, False):
            for mdl in step(form)[0]:
                mdl.free()
    torch.cuda.synchronize()
    launches0 = ig.launch_count()
    with ClockSampler(local) as clk:
        ms_b, models_b, scores_b = timed(True, steps)
    launches = (ig.launch_count() - launches0) // max(1, steps)
    ms_s, models_s, scores_s = timed(False, steps)
    identical = True
    total_tests = 0
    for w, mb, ms_, sb, ss in zip(probs, models_b, models_s, scores_b, scores_s):
        ib = mb.info()
        total_tests += nominal_tests(ib, w.test_codes.shape[0])["total"]
        for cls in (0, 1):
            identical &= all(np.array_equal(x, y) for x, y in zip(mb.patterns(cls),
                                                                   ms_.patterns(cls)))
        identical &= all(bool(torch.equal(x, y)) for x, y in zip(sb, ss))
        mb.free()
        ms_.free()
    return {"problems": len(probs), "ms_per_step": statistics.median(ms_b),
            "per_problem_ms_per_step": statistics.median(ms_s),
            "speedup_vs_per_problem": statistics.median(ms_s) / statistics.median(ms_b),
            "identical_to_per_problem": bool(identical), "tests_per_step": int(total_tests),
            "value": total_tests / (statistics.median(ms_b) * 1e-3) / 1e9, "unit": UNIT,
            "steps": steps, "gpu_launches_per_step": int(launches), "autotuned": tuned,
            "records": [int(w.train_codes.shape[0] + w.test_codes.shape[0]) for w in probs],
            "l2": "flushed before every timed step (512 MiB write)",
            "clocks": clk.summary()}


def run_batched(args, ig, torch, rank, world, local):
    """The batched workload as its own bench line."""
    from paper_2507_14222_gb300 import replicas
    r = measure_batched(args, ig, torch, local, args.steps, args.warmup,
                        replicas.replica_seed(2000, rank))
    total_ms, job_tests = replicas.job_totals(r["ms_per_step"] * args.steps,
                                              r["tests_per_step"] * args.steps, device="cuda")
    ms_per_step = total_ms / args.steps
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": job_tests / args.steps / (ms_per_step * 1e-3) / 1e9,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"ig-batched-{r['problems']}-problems",
                   "records": r["records"][:8] + ["..."], "l2": r["l2"]},
        "per_problem_launch_ms_per_step": r["per_problem_ms_per_step"],
        "speedup_vs_per_problem": r["speedup_vs_per_problem"],
        "identical_to_per_problem": r["identical_to_per_problem"],
        "autotuned": r["autotuned"], "gpu_launches": r["gpu_launches_per_step"] * args.steps,
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def measure_served(args, ig, torch, local, seed=1005):
    """Served scoring of one Poisson request stream, two ways:

    1. the continuous-batching server (ig_server_*): requests are submitted
       at their arrival times and batched as slots and memory free up;
    2. plain: one ig_score call per request, in arrival order, on one host
       thread (each request waits for the ones before it).

    The arrival rate is 0.8x the server's saturated rate (every request
    submitted at once), measured first.  Latency runs from a request's
    arrival to its results being in host memory.  Every flow's (A, N, label)
    from both ways is checked against one ig_score call over all flows."""
    import threading
    sw = igdata.served(args.served_patterns, args.served_flows, seed)
    words = [ig.ig_encode(torch.from_numpy(sw.patterns[c].view(np.int16)).cuda(), sw.cards)
             for c in (0, 1)]
    model = ig.ig_model_from_patterns(words[0], sw.support[0], words[1], sw.support[1])
    flows = ig.ig_encode(sw.flow_codes, sw.cards)              # host rows
    ref = ig.ig_score(model, torch.from_numpy(flows.view(np.int64)).cuda())
    torch.cuda.synchronize()
    ref = [t.cpu().numpy() for t in ref]
    offs = np.concatenate([[0], np.cumsum(sw.request_sizes)])
    reqs = [flows[offs[i]:offs[i + 1]] for i in range(len(sw.request_sizes))]
    server = ig.Server(model, slots=3, max_batch_flows=65536,
                       memory_budget_bytes=1 << 30)

    def run(gaps_s):
        out = [None] * len(reqs)
        tickets = [None] * len(reqs)
        t0 = time.perf_counter()

        def submitter():
            due = t0
            for i, r in enumerate(reqs):
                if gaps_s is not None:
                    due += gaps_s[i]
                    delay = due - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets[i] = server.submit(r)
        th = threading.Thread(target=submitter)
        th.start()
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0001)
            out[i] = server.wait(tickets[i])
        th.join()
        return out, time.perf_counter() - t0

    def run_plain(gaps_s):
        out, lat = [], []
        t0 = time.perf_counter()
        due = t0
        for i, r in enumerate(reqs):
            due += gaps_s[i]
            delay = due - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            A, N, lab = ig.ig_score(model, r)
            lat.append((time.perf_counter() - due) * 1e3)
            out.append((A, N, lab))
        return out, lat, time.perf_counter() - t0

    run(None)                                   # warm-up pass
    sat, sat_s = run(None)
    flows_done = int(sw.request_sizes.sum())
    sat_fps = flows_done / sat_s
    rate_req = 0.8 * sat_fps / sw.request_sizes.mean()
    gaps = sw.unit_gaps / rate_req
    b0, f0 = server.stats()
    with ClockSampler(local) as clk:
        paced, paced_s = run(gaps)
    b1, f1 = server.stats()
    lat = np.array([o[3] for o in paced])
    got = [np.concatenate([o[k] for o in paced]) for k in range(3)]
    identical = all(np.array_equal(g, r) for g, r in zip(got, ref))
    server.close()
    plain, plain_lat, plain_s = run_plain(gaps)
    got = [np.concatenate([o[k] for o in plain]) for k in range(3)]
    plain_identical = all(np.array_equal(g, r) for g, r in zip(got, ref))
    plain_lat = np.array(plain_lat)
    return {"workload": sw.name, "patterns_per_class": args.served_patterns,
            "flows": flows_done, "requests": int(len(reqs)),
            "request_sizes": "log-uniform in [1, 4096]",
            "arrivals": "Poisson at 0.8x the server's saturated rate",
            "server": {"slots": 3, "max_batch_flows": 65536, "memory_budget_bytes": 1 << 30},
            "flows_per_s": flows_done / paced_s, "seconds": paced_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "saturated_flows_per_s": sat_fps,
            "saturated_p50_ms": float(np.percentile([o[3] for o in sat], 50)),
            "batches": int(b1 - b0), "mean_flows_per_batch": (f1 - f0) / max(1, b1 - b0),
            "identical_to_one_shot": bool(identical),
            "plain": {"form": "one ig_score per request in arrival order, host buffers",
                      "flows_per_s": flows_done / plain_s, "seconds": plain_s,
                      "p50_ms": float(np.percentile(plain_lat, 50)),
                      "p99_ms": float(np.percentile(plain_lat, 99)),
                      "identical_to_one_shot": bool(plain_identical)},
            "clocks": clk.summary()}


def run_served(args, ig, torch, rank, world, local):
    """The served workload as its own bench line."""
    from paper_2507_14222_gb300 import replicas
    r = measure_served(args, ig, torch, local, replicas.replica_seed(1005, rank))
    paced_ms, job_flows = replicas.job_totals(r["seconds"] * 1e3, r["flows"], device="cuda")
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": job_flows / (paced_ms * 1e-3), "unit": "flows/s",
        "n_gpus": world, "steps": 1, "warmup": 1,
        "ms_per_step": paced_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {k: r[k] for k in ("workload", "patterns_per_class", "flows", "requests",
                                     "request_sizes", "arrivals", "server")},
        **{k: r[k] for k in ("p50_ms", "p99_ms", "saturated_flows_per_s", "saturated_p50_ms",
                             "batches", "mean_flows_per_batch", "identical_to_one_shot",
                             "plain", "clocks")},
    }
    print(json.dumps(line), flush=True)


# Stages that time exactly one kernel (the others -- split, select,
# canonical_sort, index_build -- bracket several kernels and the gaps
# between them, so they cannot stand for one kernel's roofline).
SINGLE_KERNEL_STAGES = {
    "pair_insert": "pair_insert_kernel", "compact": "compact_kernel",
    "coherence": "subset_kernel<K, ANY>", "support": "subset_kernel<K, COUNT>",
    "evidence": "subset_kernel<K, SUM>",
    "coherence_idx": "grouped_subset_kernel<K, ANY>",
    "support_idx": "grouped_subset_kernel<K, COUNT>",
    "evidence_idx": "grouped_subset_kernel<K, SUM>",
    "coherence_tc": "subset_tc_kernel<ANY>", "support_tc": "subset_tc_kernel<COUNT>",
    "evidence_tc": "subset_tc_kernel<SUM>",
}


def stage_roofline(name, ms, launches, work, info, K, clocks, steps, workload=None):
    """Roofline of one single-kernel stage over the timed steps.

    Subset-test kernels are bound by the integer pipe (LOP3 forms: 2K LOP3 per
    executed test, one per 32-bit half) or by the tensor cores (tcgen05 form:
    a 0/1 FP8 GEMM, 2 x 64K flops per executed test).  Executed tests come
    from the library: per timed stage for supports and evidence, per model
    for the coherence windows.  Memory-bound stages use byte models.
    """
    coh_idx = sum(info["coherence_tests_idx"]) * steps
    coh_tc = sum(info["coherence_tests_tc"]) * steps
    coh_dense = sum(info["coherence_tests"]) * steps - coh_idx - coh_tc
    tests = {"coherence": coh_dense, "coherence_tc": coh_tc, "coherence_idx": coh_idx}
    executed = tests.get(name, work)
    kernel = SINGLE_KERNEL_STAGES[name]
    index_tc = info.get("subset_kernel") == 4 and name.endswith("_idx")
    if index_tc:  # item-index blocks run by the fused tensor-core kernel
        kernel = kernel.replace("grouped_subset_kernel<", "subset_tc_fused_kernel<")
    out = {"kernel": kernel.replace("K,", f"{K},"), "stage": name,
           "launches": int(launches), "avg_launch_ms": ms / max(1, launches)}
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peaks = load_peaks()
    if name in ("coherence", "support", "evidence", "coherence_idx", "support_idx",
                "evidence_idx") and not index_tc:
        achieved = executed * 2 * K / (ms * 1e-3) / 1e12
        peak = LOP3_PER_SM_PER_CLK * 152 * sm_max * 1e6 / 1e12
        out.update({"tests": int(executed), "bound": "alu", "achieved": achieved,
                    "peak": peak, "unit": "Tops/s (LOP3)", "frac": achieved / peak,
                    "peak_source": f"{LOP3_PER_SM_PER_CLK} LOP3/SM/clk (measured) x 152 SMs "
                                   f"x {sm_max:.0f} MHz"})
    elif name in ("coherence_tc", "support_tc", "evidence_tc") or index_tc:
        achieved = executed * 2 * 64 * K / (ms * 1e-3) / 1e12
        bf16 = (peaks or {}).get("bf16_tflops", FALLBACK_BF16_TFLOPS)
        peak = 2.0 * bf16
        out.update({"tests": int(executed), "bound": "tensor", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s (FP8 0/1 GEMM)", "frac": achieved / peak,
                    "peak_source": ("measured bf16 burst x 2 (nominal FP8/BF16 ratio)"
                                    if peaks else "fallback bf16 x 2")})
    elif name == "pair_insert" and PROBED.get("l2_random"):
        # The dedup table (8 bytes a slot) and the records stay in L2; each
        # pair (the records of Eq. 1 included: i = j) probes one slot at a
        # hashed address and each distinct key claims one: random L2
        # accesses, rated against this GPU's measured rate of random
        # 16-byte L2 loads (ig_probe, run by this bench before timing).
        U = sum(info["n_candidates"]) * steps
        pairs = (sum(info["n_pairs"]) + sum(info["n_train"])) * steps
        acc = pairs + U
        achieved = acc / (ms * 1e-3) / 1e9
        peak = PROBED["l2_random"] / 16 / 1e9
        out.update({"bound": "l2", "achieved": achieved, "peak": peak,
                    "unit": "G random L2 accesses/s", "frac": achieved / peak,
                    "algorithmic_accesses_per_launch": acc // max(1, launches),
                    "peak_source": "measured: ig_probe L2_RANDOM (16-byte loads at random "
                                   "offsets of a 48 MiB buffer) on this GPU"})
    else:
        # Byte models (per timed step x steps) of the memory-bound stages:
        #   pair_insert (without a probed L2 rate): a hash set of K-word
        #     keys -- every pair compares its key with one stored key (8K B)
        #     and every distinct key is written once (8K B);
        #   compact: every distinct key written once (8K B).
        U = sum(info["n_candidates"]) * steps
        pairs = (sum(info["n_pairs"]) + sum(info["n_train"])) * steps
        nbytes = {"pair_insert": (pairs + U) * 8 * K, "compact": U * 8 * K}[name]
        hbm = (peaks or {}).get("hbm_gbs", FALLBACK_HBM_GBS)
        achieved = nbytes / (ms * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm,
                    "algorithmic_bytes_per_launch": nbytes // max(1, launches),
                    "peak_source": "measured" if peaks else "fallback"})
    out["traffic"] = dram_traffic(out["kernel"], workload)
    return out


# Rates measured by ig_probe on this GPU at the start of the run.
PROBED = {}


def run_probes(ig):
    """Throughput probes of the units the kernels are bound by (ig_probe):
    LOP3 rate, L2 streaming and random 16-byte loads, FP8 tcgen05 MMA rate."""
    out = {}
    for name, arg in (("lop3", 0), ("l2_read", 48), ("l2_random", 48),
                      ("mma_f8_tmem", 128), ("mma_f8_tmem", 128 | (2 << 12))):
        key = name if name != "mma_f8_tmem" or arg == 128 else "mma_f8_tmem_ring2"
        try:
            out[key] = ig.probe(name, arg)["rate"]
        except Exception as e:  # a probe that fails leaves its figure out
            out[key + "_error"] = str(e)[:120]
    PROBED.clear()
    PROBED.update({k: v for k, v in out.items() if not k.endswith("_error")})
    return out


def dram_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, or None if none was taken or the kernel's source changed since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    rec = table.get(kernel)
    if not rec:
        return None
    per = (rec.get("by_workload") or {}).get(workload)
    if per is None:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return per["bytes_per_launch"] if digest == rec["source_sha256_16"] else None


def dominant_stage(stages):
    """The single-kernel stage with the largest device time."""
    timed = [n for n, (ms, launches, _w) in stages.items()
             if n in SINGLE_KERNEL_STAGES and launches and ms > 0]
    return max(timed, key=lambda n: stages[n][0])


def roofline(stages, info, K, clocks, steps, workload=None, warm=None, warm_steps=None):
    """Rooflines of the single-kernel stages.  The headline is the dominant
    stage, timed over the timed steps (`stages`); the other stages' lines
    come from the profiled warm-up steps (`warm`) when given."""
    ref, ref_steps = (warm, warm_steps) if warm is not None else (stages, steps)
    lines = {name: stage_roofline(name, ms, launches, work, info, K, clocks, ref_steps, workload)
             for name, (ms, launches, work) in ref.items()
             if name in SINGLE_KERNEL_STAGES and launches and ms > 0}
    top = dominant_stage(stages)
    ms, launches, work = stages[top]
    head = stage_roofline(top, ms, launches, work, info, K, clocks, steps, workload)
    head["all_kernels"] = {n: {"ms_per_step": round(ref[n][0] / ref_steps, 4),
                               "frac": round(r["frac"], 4), "bound": r["bound"]}
                           for n, r in lines.items()}
    return head


def e2e_host_buffers(ig, w, tests, steps):
    """Same metric through the C ABI with numpy (host) buffers: the library
    copies codes, rows and labels in and A, N, labels (and the encoded rows)
    out inside every timed step."""
    import torch
    times = []
    h2d = d2h = 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rows = ig.ig_encode(w.train_codes, w.cards)
        test_rows = ig.ig_encode(w.test_codes, w.cards)
        model = ig.ig_fit(rows, w.train_labels)
        A, N, lab = ig.ig_score(model, test_rows)
        model.free()
        torch.cuda.synchronize()
        if i:  # the first pass is a warm-up
            times.append(time.perf_counter() - t0)
        h2d = (w.train_codes.nbytes + w.test_codes.nbytes + rows.nbytes
               + w.train_labels.nbytes + test_rows.nbytes)
        d2h = rows.nbytes + test_rows.nbytes + A.nbytes + N.nbytes + lab.nbytes
    sec = statistics.median(times)
    return {"value": tests["total"] / sec / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "s_per_step": sec}


def _oracle_pass(train_codes, train_labels, test_codes, cards, threads):
    import oracle
    rows = oracle.encode(train_codes, cards)
    test = oracle.encode(test_codes, cards)
    t0 = time.perf_counter()
    m = oracle.fit(rows, train_labels, threads=threads)
    oracle.score(m, test, threads=threads)
    sec = time.perf_counter() - t0
    nt = [int((train_labels == c).sum()) for c in (0, 1)]
    info = {"n_train": nt, "n_candidates": [m.n_candidates[0], m.n_candidates[1]],
            "n_patterns": [m.patterns[0].shape[0], m.patterns[1].shape[0]]}
    return sec, nominal_tests(info, test.shape[0])["total"]


def cpu_baseline(w):
    """The oracle as it stands, on this host's cores, over the whole workload
    once (about 10-20 s of CPU time for the 15k workload)."""
    import oracle
    threads = oracle.default_threads()
    sec, tests = _oracle_pass(w.train_codes, w.train_labels, w.test_codes, w.cards, threads)
    return {"value": tests / sec / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one full fit + score of {w.name} ({w.train_codes.shape[0]} train, "
                      f"{w.test_codes.shape[0]} test)", "seconds": sec}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    if args.workload == "served":
        return _reference_served(args, threads)
    if args.workload == "batched":
        # Bounded sample per step: the first eight problems with at most
        # 1,500 training records, each fitted and scored in full.
        probs = [w for w in (igdata.batched_problem(i) for i in range(igdata.BATCHED_PROBLEMS))
                 if w.train_codes.shape[0] <= 1500][:8]
        samples = [(w.train_codes, w.train_labels, w.test_codes, w.cards) for w in probs]
        name = f"ig-batched-{igdata.BATCHED_PROBLEMS}-problems"
        desc = (f"the first {len(probs)} batched problems with at most 1500 training records, "
                "each fitted and scored per step")
    else:
        w = igdata.WORKLOADS[args.workload]()
        # Bounded sample per step: the first 3,000 training and 1,000 test records.
        n_tr = min(3000, w.train_codes.shape[0])
        n_te = min(1000, w.test_codes.shape[0])
        samples = [(w.train_codes[:n_tr], w.train_labels[:n_tr], w.test_codes[:n_te], w.cards)]
        name = w.name
        desc = f"first {n_tr} train + {n_te} test records of {w.name} per step"
    for _ in range(args.warmup):
        for smp in samples:
            _oracle_pass(*smp, threads)
    secs, tests = [], 0
    for _ in range(args.steps):
        step_s, tests = 0.0, 0
        for smp in samples:
            sec, t = _oracle_pass(*smp, threads)
            step_s += sec
            tests += t
        secs.append(step_s)
    total = sum(secs)
    _print_reference(args, world, tests * args.steps / total / 1e9, UNIT,
                     total / args.steps * 1e3, name, desc, threads)


def _reference_served(args, threads):
    """The oracle scoring a bounded sample of the served workload's flows
    against its full pattern sets (the model is built once, untimed)."""
    import oracle
    sw = igdata.served(args.served_patterns, args.served_flows, 1005)
    om = oracle.model_from_patterns({c: oracle.encode(sw.patterns[c], sw.cards) for c in (0, 1)},
                                    sw.support)
    m = min(2000, sw.flow_codes.shape[0])
    flows = oracle.encode(sw.flow_codes[:m], sw.cards)
    for _ in range(args.warmup):
        oracle.score(om, flows, threads)
    total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.score(om, flows, threads)
        total += time.perf_counter() - t0
    desc = f"first {m} flows of {sw.name} scored per step (one-shot, all patterns)"
    _print_reference(args, 1, m * args.steps / total, "flows/s", total / args.steps * 1e3,
                     sw.name, desc, threads)


def _print_reference(args, world, value, unit, ms_per_step, name, desc, threads):
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": name, "sample": desc},
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
