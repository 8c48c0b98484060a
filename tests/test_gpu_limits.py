"""The bounded device-side waits return IM_E_TIMEOUT instead of holding the GPU.

Every loop of the device code that waits or iterates is bounded: the grid
barrier between the levels of a cooperative phase launch (barrier_wait_ns of
global time) and the levels of one phase (max_levels).  These tests make each
bound run out on a tiny graph with im_ctx_set_limits, check that the call
returns IM_E_TIMEOUT with the matching message, and that the context then
works again: the next call, with the default limits, gives the oracle's result.
No test faults, traps or hangs the GPU: the waits give up by themselves.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TIMEOUT = -5


@pytest.fixture(scope="module")
def im():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as lib
    lib.load_library()
    return lib


def _path(n=300):
    # a long path with p = 1: the registers need about one level per hop
    return W.from_edges(n, [(i, i + 1) for i in range(n - 1)])


def _check_build(im, G, g, model, J=64, seed=7):
    sk = im.im_sketch_build(G, J, seed)
    X, salt = O.draw_sims(seed, J)
    assert np.array_equal(sk.registers(), O.build_reverse(g, O.thresholds(g, model), J, X, salt))


def _check_select(im, G, g, model, J=64, K=4, seed=7):
    r = im.im_select_seeds(G, K, J, seed=seed)
    ref = O.select_seeds(g, O.thresholds(g, model), J, K, seed, 0.01, "reverse")
    assert r["seeds"].tolist() == ref["seeds"].tolist()
    assert np.array_equal(r["score"], ref["score"])


@pytest.mark.parametrize("persistent", [1, 0])
def test_level_limit_times_out_and_the_context_recovers(im, persistent):
    g = _path()
    model = {"kind": "uniform", "p": 1.0}
    ctx = im.im_ctx_create(0)
    im.im_ctx_set_tuning(ctx, {"persistent": persistent})
    G = im.im_graph_load(ctx, g.rowptr, g.col, model)
    im.im_ctx_set_limits(ctx, max_levels=2)
    for call in (lambda: im.im_sketch_build(G, 64, 7), lambda: im.im_select_seeds(G, 4, 64, seed=7)):
        with pytest.raises(im.IMError) as ei:
            call()
        assert ei.value.status == TIMEOUT
        assert "did not empty" in str(ei.value)
    im.im_ctx_set_limits(ctx)  # defaults
    _check_build(im, G, g, model)
    _check_select(im, G, g, model)


def test_barrier_wait_limit_times_out_and_the_context_recovers(im):
    g = W.erdos_renyi(3000, 24000, seed=3)
    model = {"kind": "uniform", "p": 0.3}
    ctx = im.im_ctx_create(0)
    im.im_ctx_set_tuning(ctx, {"persistent": 1})
    G = im.im_graph_load(ctx, g.rowptr, g.col, model)
    # 0 ns: a block that has to wait at the first grid barrier gives up at once
    im.im_ctx_set_limits(ctx, barrier_wait_ns=0)
    for call in (lambda: im.im_sketch_build(G, 64, 7), lambda: im.im_select_seeds(G, 4, 64, seed=7)):
        with pytest.raises(im.IMError) as ei:
            call()
        assert ei.value.status == TIMEOUT
        assert "barrier" in str(ei.value)
    im.im_ctx_set_limits(ctx)
    _check_build(im, G, g, model)
    _check_select(im, G, g, model)
    # a limit well above a level's duration changes nothing
    im.im_ctx_set_limits(ctx, barrier_wait_ns=500_000_000, max_levels=1000)
    _check_select(im, G, g, model)


def test_limits_reject_out_of_range_levels(im):
    ctx = im.im_ctx_create(0)
    for bad in (0, -1, 16383):
        with pytest.raises(im.IMError) as ei:
            im.im_ctx_set_limits(ctx, max_levels=bad)
        assert ei.value.status == -1
