"""Parity at the large workload (R-MAT scale 24 ef 16, trivalency IC, J=512,
K=50: 16.7M vertices, 263M edges, 8.6 GB of registers): seeds, scores and
estimates against the oracle's stored run (tests/golden/make_golden.py), the
final registers by digest, and sampled registers of a fresh build (one
oracle search each)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as im
    wl = W.workload("rmat24")
    g = wl.graph()
    gold = json.load(open(os.path.join(GOLDEN, "select_rmat24.json")))
    h = hashlib.sha256()
    h.update(g.rowptr.tobytes())
    h.update(g.col.tobytes())
    assert h.hexdigest() == gold["graph_sha256"], "generator output differs from the golden run"
    ctx = im.im_ctx_create(0)
    G = im.im_graph_load(ctx, g.rowptr, g.col, wl.model)
    return im, ctx, G, g, wl, gold


def test_large_workload_selection_matches_oracle(setup):
    im, ctx, G, g, wl, gold = setup
    r = im.im_select_seeds(G, wl.K, wl.J, seed=wl.seed, rebuild_eps=wl.rebuild_eps, return_sketch=True)
    assert r["seeds"].tolist() == gold["seeds"]
    assert r["score"].tolist() == gold["score"]
    np.testing.assert_allclose(r["est"], [float.fromhex(x) for x in gold["est"]], rtol=1e-12, atol=0)
    assert im.im_last_stats(ctx)["builds"] == 1 + gold["rebuilds"]
    sk = r["sketch"]
    M = sk.registers()
    assert int(np.count_nonzero(M == 0xFF)) == gold["visited"]
    assert hashlib.sha256(M.tobytes()).hexdigest() == gold["registers_sha256"]
    del M
    sk.free()


def test_large_workload_build_sampled_registers(setup):
    im, ctx, G, g, wl, gold = setup
    sk = im.im_sketch_build(G, wl.J, wl.seed)
    M = sk.registers()
    X, salt = sk.sims()
    sk.free()
    thr = O.thresholds(g, wl.model)
    rng = np.random.default_rng(24)
    deg = np.diff(g.rowptr)
    us = np.concatenate([rng.integers(0, g.n, 6), np.argsort(deg)[-3:]])
    for u in us:
        j = int(rng.integers(0, wl.J))
        assert M[u, j] == O.register_entry(g, thr, X[j], salt[j], int(u)), (u, j)
    # the live-edge invariant on a sample of edges: M[u][j] >= M[v][j] when
    # (u, v) is live in simulation j (registers are max-merged along live edges)
    js = rng.integers(0, wl.J, 4)
    es = rng.integers(0, g.m, 4000)
    src = np.searchsorted(g.rowptr, es, side="right") - 1
    dst = g.col[es]
    for j in js:
        mark = np.array([(int(X[j]) ^ O.edge_hash(int(s), int(d))) < int(thr[e])
                         for e, s, d in zip(es, src, dst)])
        assert mark.any()
        assert np.all(M[src[mark], j] >= M[dst[mark], j])
