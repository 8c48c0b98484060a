"""Schedule autotuner for the frontier kernels.

Chooses the im_tuning knobs (vertex-to-warp mapping: the in-degree above which
a hub is pushed by per-simulation hash search instead of an in-edge scan;
work granularity: 32-edge batches per claimed unit; frontier thresholds: when a
propagation level walks every vertex in vertex order, and below which level
size queues switch from vertices to (vertex, chunk) buckets) by timing short
runs of the caller's workload.  The knobs change how work is split, never a
result.
"""
from __future__ import annotations

import itertools
import json
import os
import time

from . import im_ctx_get_tuning, im_ctx_set_tuning

DEFAULT_SPACE = {
    "heavy_indeg": [64, 256],
    "light_batches": [4, 16, 32],
    "dense_div": [0, 2],
    "buckets": [0, 1, 2],
}


def candidates(space: dict | None = None):
    space = space or DEFAULT_SPACE
    keys = sorted(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        yield dict(zip(keys, vals))


def tune(ctx, run, space: dict | None = None, repeats: int = 2, cache: str | None = None,
         key: str | None = None) -> dict:
    """Time `run()` (a callable doing one representative unit of work) under
    every candidate tuning; keep the fastest on `ctx` and return a report.
    With `cache` (a JSON path) and `key`, a stored choice is reused."""
    if cache and key and os.path.exists(cache):
        stored = json.load(open(cache)).get(key)
        if stored:
            im_ctx_set_tuning(ctx, stored["tuning"])
            return dict(stored, cached=True)
    base = im_ctx_get_tuning(ctx)
    trials = []
    for cand in candidates(space):
        t = dict(base, **cand)
        im_ctx_set_tuning(ctx, t)
        run()  # warm-up under this schedule
        best = float("inf")
        for _ in range(repeats):
            t0 = time.perf_counter()
            run()
            best = min(best, time.perf_counter() - t0)
        trials.append({"tuning": cand, "ms": best * 1e3})
    winner = min(trials, key=lambda x: x["ms"])
    im_ctx_set_tuning(ctx, dict(base, **winner["tuning"]))
    report = {"tuning": dict(base, **winner["tuning"]), "ms": winner["ms"], "trials": trials}
    if cache and key:
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[key] = {"tuning": report["tuning"], "ms": report["ms"]}
        json.dump(data, open(cache, "w"), indent=1)
    return report
