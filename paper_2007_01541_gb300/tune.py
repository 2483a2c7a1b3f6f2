"""Measurement-driven choice of the mixed-precision factorization's schedule.

Per elimination-tree level the pivot columns can run as one launch of
dependency-ordered tasks (small per-step latency, but every task of the level
holds an SM while it waits) or as a (panel, update) launch pair per 64-column
pivot block (no waiting, but a launch gap per step).  Which is faster depends
on the level's shape: how many fronts, how wide, how tall.  tune_schedule()
times whole factorizations of the caller's matrix on the caller's GPU and
chooses the flags level by level (coordinate descent from the all-tasks
schedule, deepest level first, a change kept only if it saves more than
`min_gain` of the time), then leaves the solver on the chosen schedule.

The choice is cached in a JSON file keyed by the analysis (order, stored
entries, supernodes, levels, ordering and amalgamation options) and the
device name, so a second run on the same structure applies it without
measuring.  Both schedules compute the same factor; only the time differs.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "schedule_cache.json")


def _device_name() -> str:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        pass
    return "unknown"


def structure_key(solver, extra: str = "") -> str:
    """Key of the cached choice: the analysis' shape and options, the device."""
    i = solver.info()
    sym = solver.symbolic()
    h = hashlib.sha1()
    for f in ("n", "nnz_A_lower", "nnz_L", "nsuper", "nlevels", "max_front", "max_width"):
        h.update(str(int(i[f])).encode())
    h.update(sym["super_first"].tobytes())
    h.update(sym["super_rowptr"].tobytes())
    h.update(repr(solver.options).encode())
    h.update(_device_name().encode())
    h.update(extra.encode())
    return h.hexdigest()


def _time_factor(solver, values, reps: int) -> float:
    solver.factor(values, "mixed")            # graph capture and warm-up
    best = float("inf")
    for _ in range(reps):
        t = time.perf_counter()
        solver.factor(values, "mixed")        # synchronous: reads the status word
        best = min(best, time.perf_counter() - t)
    return best * 1e3


def tune_schedule(solver, values, reps: int = 5, min_gain: float = 0.003, cache_path: str | None = DEFAULT_CACHE,
                  extra_key: str = "") -> dict:
    """Choose the per-level schedule of `solver` (analyzed) for `values` by
    timing mixed-precision factorizations; returns {"schedule", "ms",
    "ms_default", "cached", "evaluations"} and leaves the solver on the
    chosen schedule."""
    key = structure_key(solver, extra_key)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    hit = cache.get(key)
    nlev = solver.info()["nlevels"]
    if hit and len(hit.get("schedule", [])) == nlev:
        solver.set_level_schedule(hit["schedule"])
        return dict(hit, cached=True)
    best = [0] * nlev
    solver.set_level_schedule(best)
    t_best = t_default = _time_factor(solver, values, reps)
    evals = 1
    for lev in range(nlev):
        cand = list(best)
        cand[lev] = 1
        solver.set_level_schedule(cand)
        t = _time_factor(solver, values, reps)
        evals += 1
        if t < t_best * (1.0 - min_gain):
            best, t_best = cand, t
    solver.set_level_schedule(best)
    out = {"schedule": best, "ms": t_best, "ms_default": t_default, "evaluations": evals,
           "device": _device_name()}
    if cache_path:
        cache[key] = out
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(out, cached=False)
