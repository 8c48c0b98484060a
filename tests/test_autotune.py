"""The schedule autotuner's host logic on CPU: every candidate of the space is
tried, the fastest is kept on the context, and a cached choice is reused.  The
context calls and the clock are replaced by fakes (no GPU)."""
import itertools
import json

import pytest

from paper_2410_14047_gb300 import autotune as A

BASE = {"heavy_indeg": 256, "light_batches": 4, "grid_blocks": 0, "check_every": 2, "persistent": 1,
        "dense_div": 0, "lazy_pick": 1, "buckets": 2, "incremental": 1, "chain": 8, "pick_tile": 4,
        "dense_out": 1, "dense_all": 0}


class FakeCtx:
    def __init__(self):
        self.tuning = dict(BASE)
        self.sets = 0


@pytest.fixture
def fake(monkeypatch):
    clock = {"t": 0.0}

    def get(ctx):
        return dict(ctx.tuning)

    def put(ctx, t):
        ctx.tuning = dict(t)
        ctx.sets += 1

    monkeypatch.setattr(A, "im_ctx_get_tuning", get)
    monkeypatch.setattr(A, "im_ctx_set_tuning", put)
    monkeypatch.setattr(A.time, "perf_counter", lambda: clock["t"])
    return clock


def cost(t):
    # a schedule-dependent run time with one best point in the default space
    return (1.0 + 0.1 * abs(t["light_batches"] - 16) + 0.2 * (t["dense_div"] != 2)
            + 0.05 * (t["heavy_indeg"] == 256) + 0.3 * (t["buckets"] == 0) + 0.01 * (t["pick_tile"] != 2)
            + 0.02 * (t["dense_out"] != 0) + 0.03 * (t["dense_all"] != 3))


def test_every_candidate_is_tried_and_the_fastest_kept(fake):
    ctx = FakeCtx()

    def run():
        fake["t"] += cost(ctx.tuning)

    rep = A.tune(ctx, run, repeats=2)
    space = A.DEFAULT_SPACE
    n = 1
    for v in space.values():
        n *= len(v)
    # the frontier knobs together, then the dense output, then the J-tile width
    assert len(rep["trials"]) == n + 8 + len(A.DEFAULT_STAGES[2]["pick_tile"])
    tried = [tuple(sorted(tr["tuning"].items())) for tr in rep["trials"][:n]]
    assert len(set(tried)) == n
    best = min(candidates_with_cost(space), key=lambda x: x[1])[0]
    for k, v in best.items():
        assert ctx.tuning[k] == v and rep["tuning"][k] == v
    for tr in rep["trials"][n:]:
        assert {k: tr["tuning"][k] for k in best} == best
    for tr in rep["trials"][n + 8:]:
        assert tr["tuning"]["dense_out"] == 0 and tr["tuning"]["dense_all"] == 3
    assert ctx.tuning["pick_tile"] == 2 and rep["tuning"]["pick_tile"] == 2
    assert ctx.tuning["dense_out"] == 0 and ctx.tuning["dense_all"] == 3
    # knobs outside the space keep the context's values
    for k in ("grid_blocks", "check_every", "persistent", "lazy_pick", "incremental", "chain"):
        assert ctx.tuning[k] == BASE[k]
    assert rep["ms"] == pytest.approx(cost(dict(BASE, **best, pick_tile=2, dense_out=0, dense_all=3)) * 1e3)


def candidates_with_cost(space):
    keys = sorted(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        t = dict(zip(keys, vals))
        yield t, cost(dict(BASE, **t))


def test_cached_choice_is_reused(fake, tmp_path):
    ctx = FakeCtx()
    calls = {"n": 0}

    def run():
        calls["n"] += 1
        fake["t"] += cost(ctx.tuning)

    cache = str(tmp_path / "tune.json")
    space = {"light_batches": [4, 16], "dense_div": [0, 2]}
    first = A.tune(ctx, run, space=space, repeats=1, cache=cache, key="g1")
    assert calls["n"] == 2 * 4 and not first.get("cached")
    stored = json.load(open(cache))["g1"]
    assert stored["tuning"]["light_batches"] == 16 and stored["tuning"]["dense_div"] == 2
    ctx2 = FakeCtx()
    again = A.tune(ctx2, run, space=space, repeats=1, cache=cache, key="g1")
    assert again["cached"] and calls["n"] == 8  # no further runs
    assert ctx2.tuning["light_batches"] == 16 and ctx2.tuning["dense_div"] == 2
    # another key tunes afresh and keeps the first entry
    A.tune(FakeCtx(), run, space=space, repeats=1, cache=cache, key="g2")
    assert set(json.load(open(cache))) == {"g1", "g2"}
