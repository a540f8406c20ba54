"""Autotuner for the subset-test form and the item-index tiling.

Every choice gives the same results; they differ only in speed, which
depends on the word count K, the number of records and how sparse the
records are.  The tuner groups problems by (K rounded up to a power of two,
log2 of the record count), times each candidate configuration on one
representative problem per group (fit + score, after a warm-up run), and
keeps the fastest.  Choices are cached in a JSON file keyed by the GPU name,
its SM count and the group, so that a batch of problems is tuned once per
machine: $IG_AUTOTUNE_CACHE, or _build/autotune.json beside the library.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import buildlib as _build

# Candidate configurations: the item index with several block shapes and
# orientation policies, the item index on the tensor cores, the tensor-core
# GEMM, and the plain integer kernel.
CANDIDATES = [
    {"subset_kernel": 3, "index_max_q": 4, "index_flip_factor": 2},
    {"subset_kernel": 3, "index_max_q": 2, "index_flip_factor": 2},
    {"subset_kernel": 3, "index_max_q": 1, "index_flip_factor": 2},
    {"subset_kernel": 3, "index_max_q": 4, "index_flip_factor": 1},
    {"subset_kernel": 3, "index_max_q": 4, "index_flip_factor": 1 << 20},
    {"subset_kernel": 4},
    {"subset_kernel": 2},
    {"subset_kernel": 1},
]


def bucket(K: int, n: int) -> str:
    kt = 1
    while kt < K:
        kt *= 2
    return f"kt{kt}-n2^{int(round(math.log2(max(n, 1))))}"


def _default_path() -> str:
    return os.environ.get("IG_AUTOTUNE_CACHE", os.path.join(_build.BUILD, "autotune.json"))


class Autotuner:
    def __init__(self, path: str | None = None):
        self.path = path or _default_path()
        try:
            with open(self.path) as f:
                self.cache = json.load(f)
        except (OSError, ValueError):
            self.cache = {}
        self.timings = {}

    @staticmethod
    def _device_key() -> str:
        import torch
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.name}/{p.multi_processor_count}sm"

    def _key(self, K: int, n: int) -> str:
        return f"{self._device_key()}/{bucket(K, n)}"

    def _save(self):
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def tune(self, problems, candidates=None, repeats: int = 2, retune: bool = False) -> dict:
        """problems: [(rows, labels, test_rows)] with CUDA tensors.

        Returns {group: config} for the groups present.
        """
        import torch

        from . import ig_fit, ig_score
        candidates = candidates or CANDIDATES
        groups = {}
        for prob in problems:
            n, K = int(prob[0].shape[0]), int(prob[0].shape[1])
            groups.setdefault(self._key(K, n), []).append(prob)
        for key, probs in groups.items():
            if key in self.cache and not retune:
                continue
            probs = sorted(probs, key=lambda p: int(p[0].shape[0]))
            rows, labels, test = probs[len(probs) // 2]
            best = None
            for cand in candidates:
                times = []
                for rep in range(repeats + 1):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    model = ig_fit(rows, labels, **cand)
                    ig_score(model, test)
                    torch.cuda.synchronize()
                    if rep:
                        times.append(time.perf_counter() - t0)
                    model.free()
                t = min(times)
                self.timings.setdefault(key, {})[json.dumps(cand, sort_keys=True)] = t
                if best is None or t < best[0]:
                    best = (t, cand)
            self.cache[key] = best[1]
        self._save()
        return {k: self.cache[k] for k in groups}

    def config_for(self, K: int, n: int) -> dict | None:
        return self.cache.get(self._key(K, n))

    def params_for(self, K: int, n: int):
        from . import make_params
        cfg = self.config_for(K, n)
        return make_params(**cfg) if cfg else None
