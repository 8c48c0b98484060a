"""Batched form: many graphs in one device union; each graph's result must be
identical to its solo run (same seed, J, K, rebuild threshold), and the solo
runs are checked against the oracle for a few graphs."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def im():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2410_14047_gb300 as lib
    lib.load_library()
    return lib


def _mix(seed):
    rng = np.random.default_rng(seed)
    graphs, p, J, K = [], [], [], []
    for i in range(14):
        n = int(rng.integers(200, 6000))
        kind = i % 3
        if kind == 0:
            g = W.chung_lu(n, float(rng.uniform(4, 16)), 2.1, seed=100 + i)
        elif kind == 1:
            g = W.erdos_renyi(n, int(n * rng.uniform(2, 8)), seed=100 + i)
        else:
            g = W.rmat(int(np.log2(n)) + 1, 8, seed=100 + i)
        graphs.append(g)
        p.append(float(np.float32(rng.uniform(0.005, 0.3))))
        J.append(int(rng.choice([16, 64, 128])))
        K.append(int(min(g.n, rng.integers(1, 12))))
    return graphs, p, J, K


@pytest.mark.parametrize("eps", [0.01, -1.0])
def test_batch_equals_solo_runs(im, eps):
    graphs, p, J, K = _mix(7)
    ctx = im.im_ctx_create(0)
    B = im.im_batch_load(ctx, graphs, p)
    res = im.im_batch_select_seeds(B, J, K, seed=99, rebuild_eps=eps)
    for g, pg, Jg, Kg, r in zip(graphs, p, J, K, res):
        G = im.im_graph_load(ctx, g.rowptr, g.col, {"kind": "uniform", "p": pg})
        solo = im.im_select_seeds(G, Kg, Jg, seed=99, rebuild_eps=eps)
        assert r["seeds"].tolist() == solo["seeds"].tolist()
        assert np.array_equal(r["score"], solo["score"])
        np.testing.assert_allclose(r["est"], solo["est"], rtol=1e-12, atol=0)


def test_batch_against_oracle(im):
    graphs, p, J, K = _mix(11)
    ctx = im.im_ctx_create(0)
    im.im_ctx_set_tuning(ctx, {"heavy_indeg": 8})
    B = im.im_batch_load(ctx, graphs, p)
    res = im.im_batch_select_seeds(B, J, K, seed=5)
    for i in (0, 4, 9, 13):
        g = graphs[i]
        ref = O.select_seeds(g, O.thresholds(g, {"kind": "uniform", "p": p[i]}), J[i], K[i], 5, 0.01, "reverse")
        assert res[i]["seeds"].tolist() == ref["seeds"].tolist()
        assert np.array_equal(res[i]["score"], ref["score"])


def test_per_target_model_against_oracle(im):
    # the per-target model the batched form runs on (every edge into v fires
    # with w[v]), loaded on its own with uneven w, against the oracle's
    # per-target thresholds
    ctx = im.im_ctx_create(0)
    rng = np.random.default_rng(23)
    for g in (W.chung_lu(3000, 10.0, 2.1, seed=41), W.rmat(11, 12, seed=42)):
        w = rng.uniform(0.0, 0.4, g.n).astype(np.float32)
        model = {"kind": "target", "w": w}
        G = im.im_graph_load(ctx, g.rowptr, g.col, model)
        for J, K in ((64, 6), (128, 4)):
            r = im.im_select_seeds(G, K, J, seed=31, return_sketch=True)
            ref = O.select_seeds(g, O.thresholds(g, model), J, K, 31, 0.01, "reverse")
            assert r["seeds"].tolist() == ref["seeds"].tolist()
            assert np.array_equal(r["score"], ref["score"])
            assert np.array_equal(r["sketch"].registers(), ref["M"])


def test_every_batched_graph_against_oracle_per_target_thresholds(im):
    # the whole batch (every graph, not a sample) against the oracle run with
    # the per-target thresholds the batch uses: w[v] = p of v's graph
    graphs, p, J, K = _mix(17)
    ctx = im.im_ctx_create(0)
    B = im.im_batch_load(ctx, graphs, p)
    res = im.im_batch_select_seeds(B, J, K, seed=8)
    for i, g in enumerate(graphs):
        thr = O.thresholds(g, {"kind": "target", "w": np.full(g.n, p[i], np.float32)})
        ref = O.select_seeds(g, thr, J[i], K[i], 8, 0.01, "reverse")
        assert res[i]["seeds"].tolist() == ref["seeds"].tolist(), i
        assert np.array_equal(res[i]["score"], ref["score"]), i
        np.testing.assert_allclose(res[i]["est"], ref["est"], rtol=1e-12, atol=0)
