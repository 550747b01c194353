"""Autotuner of the planner parameters (bin thresholds, table load, threads
per row, dense-row thresholds) for one workload.

Coordinate search: starting from the defaults, each parameter in turn takes
each of its candidate values while the others stay at the best so far; a
candidate is kept when the full product (symbolic + numeric, CUDA events)
gets faster. None of the parameters changes the result. Results are cached in
a JSON file keyed by GPU name and SM count, then by a workload key. The
batched kernel's table size has its own tuner in the library
(smash_batched_autotune).
"""
from __future__ import annotations

import json
import os

SPACE = [
    ("group_shift", [3, 4, 5]),
    ("max_load", [0.5, 0.7]),
    ("dense_ratio", [2, 4, 8, 16]),
    ("sym_dense_ratio", [16, 64, 256]),
    ("bitmap_ratio", [1, 4, 16]),
    ("dense_blocks", [1, 2, 4]),
    ("dense_owner", [0, 1]),
    ("row_window_tbits", [6, 7, 8]),
]


def gpu_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def _time(handle, dA, dB, reps: int = 2) -> float:
    import torch
    s = torch.cuda.current_stream()
    handle.spgemm(dA, dB, s)          # warm (workspace growth)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        handle.spgemm(dA, dB, s)
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(handle, dA, dB, workload_key: str, cache_path: str | None = None, reps: int = 2):
    """Best parameters for C = A*B (applied to the handle); returns (params, ms)."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    gk = gpu_key()
    hit = cache.get(gk, {}).get(workload_key)
    if hit:
        handle.set_params(**hit["params"])
        return hit["params"], hit["ms"]
    base = handle.params.as_dict()
    best = dict(base)
    handle.set_params(**best)
    best_ms = _time(handle, dA, dB, reps)
    for name, values in SPACE:
        for v in values:
            if best.get(name) == v:
                continue
            trial = dict(best)
            trial[name] = v
            handle.set_params(**trial)
            ms = _time(handle, dA, dB, reps)
            if ms < best_ms * 0.98:
                best, best_ms = trial, ms
    handle.set_params(**best)
    out = {k: best[k] for k, _ in SPACE}
    if cache_path:
        cache.setdefault(gk, {})[workload_key] = {"params": out, "ms": best_ms}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return out, best_ms
