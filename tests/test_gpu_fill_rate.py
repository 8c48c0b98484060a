"""Warp fill-rate diagnostic (Table 6 analogue): the GPU's counts of live
(edge, simulation) pairs and of the 32-simulation warps that hold them, in
draw order and in sorted-X order, against the same counts taken on the host
from the oracle's hash, threshold and SplitMix64 routines."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _host_counts(g, model, J, seed):
    thr = O.thresholds(g, model).astype(np.int64)
    raw = O.splitmix64(seed, J)
    X = (raw & np.uint64(0x7FFFFFFF)).astype(np.int64)
    order = np.argsort(X, kind="stable")           # sorted position -> draw index
    pos = np.empty(J, dtype=np.int64)
    pos[order] = np.arange(J)                       # draw index -> sorted position
    live = wd = ws = 0
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    for e in range(g.m):
        h = O.edge_hash(int(src[e]), int(g.col[e]))
        lv = np.nonzero((X ^ h) < thr[e])[0]        # live draw indices
        live += lv.size
        wd += np.unique(lv >> 5).size
        ws += np.unique(pos[lv] >> 5).size
    return g.m, live, wd, ws


@pytest.mark.parametrize("model,J", [({"kind": "uniform", "p": 0.01}, 256), ({"kind": "uniform", "p": 0.1}, 64),
                                     ({"kind": "wc"}, 128), ({"kind": "trivalency", "seed": 3}, 256)])
def test_fill_rate_counts_match_host(model, J):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as im
    g = W.erdos_renyi(1500, 9000, seed=12)
    ctx = im.im_ctx_create(0)
    G = im.im_graph_load(ctx, g.rowptr, g.col, model)
    r = im.im_fill_rate(G, J, seed=77)
    m, live, wd, ws = _host_counts(g, model, J, 77)
    assert (r["edges"], r["live"], r["warps_draw"], r["warps_sorted"]) == (m, live, wd, ws)
    assert r["candidates"] >= r["live"]
