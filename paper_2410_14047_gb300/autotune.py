"""Schedule autotuner for the frontier kernels.

Chooses the im_tuning knobs (vertex-to-warp mapping: the in-degree above which
a hub is pushed by per-simulation hash search instead of an in-edge scan;
work granularity: 32-edge batches per claimed unit; frontier thresholds: when a
propagation level walks every vertex in vertex order, and below which level
size queues switch from vertices to (vertex, chunk) buckets, whether dense
walks skip building queues and push every live simulation; J-tile width: the 16-simulation register pieces
one lane sums per row in the estimate + argmax pass) by timing short runs of
the caller's workload.  The frontier knobs are tried together (every
combination), then the dense-walk output with them fixed, then the J-tile
width (the estimate pass does not interact with the frontier schedule).
The knobs change how work is split, never a result.
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


# stages of the default search: each stage's combinations are timed with the
# winners of the earlier stages in place
# (dense_all: bit 0 = propagation walks, bit 1 = cover walks push every
# live / visited simulation)
DEFAULT_STAGES = [DEFAULT_SPACE, {"dense_out": [0, 1], "dense_all": [0, 1, 2, 3]}, {"pick_tile": [1, 2, 4]}]


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
    stages = DEFAULT_STAGES if space is None else [space]
    trials = []
    chosen = {}
    winner = None
    for stage in stages:
        stage_trials = []
        for cand in candidates(stage):
            pick = dict(chosen, **cand)
            im_ctx_set_tuning(ctx, dict(base, **pick))
            run()  # warm-up under this schedule
            best = float("inf")
            for _ in range(repeats):
                t0 = time.perf_counter()
                run()
                best = min(best, time.perf_counter() - t0)
            stage_trials.append({"tuning": pick, "ms": best * 1e3})
        winner = min(stage_trials, key=lambda x: x["ms"])
        chosen = dict(winner["tuning"])
        trials += stage_trials
    im_ctx_set_tuning(ctx, dict(base, **chosen))
    report = {"tuning": dict(base, **chosen), "ms": winner["ms"], "trials": trials}
    if cache and key:
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[key] = {"tuning": report["tuning"], "ms": report["ms"]}
        json.dump(data, open(cache, "w"), indent=1)
    return report
