"""Autotuner for the RANSAC launch shape (block size, hypotheses per thread,
correspondences per work item).

Candidates are timed on the caller's actual batch: each is captured into a
CUDA graph and replayed, timed with CUDA events; the fastest wins.  Results
are cached in a small JSON file keyed by (GPU name, SM count, workload
bucket) so later plans of a similar shape skip the sweep.  The launch shape
never changes results (the scoring is exact integer counting per
hypothesis), so tuning is safe at any time.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

_lock = threading.Lock()

CANDIDATES = [
    dict(block_warps=w, hyps_per_thread=h, tile_points=t)
    for w in (4, 8, 16)
    for h in (1, 2, 4)
    for t in (256, 512, 1024, 2048, 4096)
    if h <= w
]


def cache_path() -> str:
    return os.environ.get("ACA_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))


def _bucket(P: int, total_points: int, total_hyps: int) -> str:
    lg = lambda x: int(round(math.log2(max(1, x))))
    return f"P{lg(P)}-N{lg(total_points / max(1, P))}-K{lg(total_hyps / max(1, P))}"


def _key(device, P, total_points, total_hyps, tag="") -> str:
    props = torch.cuda.get_device_properties(device)
    return f"{props.name}|{props.multi_processor_count}|{_bucket(P, total_points, total_hyps)}" + (f"|{tag}" if tag else "")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(cache):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_plan(plan, reps: int = 10) -> float:
    """Average ms of one graph replay of `plan` (captured here)."""
    plan.capture(warmup=1)
    for _ in range(2):
        plan.graph.replay()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan.graph.replay()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(make_plan, P: int, total_points: int, total_hyps: int, device=None, candidates=None, reps: int = 10,
         use_cache: bool = True, tag: str = ""):
    """Return (best_params, {str(params): ms}).  make_plan(**params) builds a
    RansacPlan for the workload with the given launch parameters; `tag`
    separates cache entries of different plan kinds (e.g. the adaptive stop)
    for the same workload shape."""
    device = device if device is not None else torch.cuda.current_device()
    key = _key(device, P, total_points, total_hyps, tag)
    with _lock:
        cache = _load() if use_cache else {}
        if key in cache:
            return cache[key]["params"], cache[key].get("timings", {})
    timings = {}
    best, best_ms = None, float("inf")
    for cand in (candidates or CANDIDATES):
        ms = time_plan(make_plan(**cand), reps)
        timings[json.dumps(cand, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    with _lock:
        cache = _load()
        cache[key] = {"params": best, "ms": best_ms, "timings": timings}
        _store(cache)
    return best, timings
