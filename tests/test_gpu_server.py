"""Served form: concurrent queries on resident graphs (im_server_*).

Each query's result must be the same alone (a plain im_select_seeds call) and
in the mix (run by the server while other queries overlap on the device), and
admission must keep the reserved device bytes within the budget."""
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


@pytest.fixture(scope="module")
def resident(im):
    ctx = im.im_ctx_create(0)
    graphs = [W.rmat(11, 8, seed=3), W.rmat(13, 16, seed=4), W.erdos_renyi(3000, 24000, seed=5),
              W.chung_lu(5000, 12.0, 2.1, seed=6)]
    loaded = [im.im_graph_load(ctx, g.rowptr, g.col, {"kind": "wc"}) for g in graphs]
    return ctx, graphs, loaded


def _queries(n_graphs, count, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(count):
        model = {"kind": "uniform", "p": 0.05} if rng.integers(2) else {"kind": "wc"}
        if i % 5 == 4:
            model = {"kind": "trivalency", "seed": 77}
        qs.append(dict(graph=int(rng.integers(n_graphs)), K=int(rng.choice([1, 5, 10, 25])),
                       J=int(rng.choice([16, 64, 256, 1024])), model=model, seed=int(rng.integers(1 << 40)),
                       rebuild_eps=float(rng.choice([0.01, -1.0, 0.2]))))
    return qs


def _solo(im, loaded, q):
    return im.im_select_seeds(loaded[q["graph"]], q["K"], q["J"], model=q["model"], seed=q["seed"],
                              rebuild_eps=q["rebuild_eps"])


def _same(a, b):
    assert a["seeds"].tolist() == b["seeds"].tolist()
    assert np.array_equal(a["score"], b["score"])
    np.testing.assert_allclose(a["est"], b["est"], rtol=1e-12, atol=0)


def test_served_results_equal_solo_runs(im, resident):
    _, graphs, loaded = resident
    qs = _queries(len(loaded), 24, seed=1)
    solo = [_solo(im, loaded, q) for q in qs]
    srv = im.Server(0, slots=6)
    try:
        ids = [srv.add_graph(G) for G in loaded]
        assert ids == list(range(len(loaded)))
        tickets = [srv.submit(**q) for q in qs]  # all arrive at once: the slots fill up
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for q, r, s in zip(qs, res, solo):
        assert r["status"] == 0, r["error"]
        _same(r, s)
        assert r["t_submit_ms"] <= r["t_start_ms"] <= r["t_done_ms"]
    assert st["completed"] == len(qs) and st["failed"] == 0
    assert st["running_peak"] >= 2  # queries overlapped
    assert st["reserved"] == 0 and st["running"] == 0 and st["pending"] == 0


def test_served_results_match_oracle(im, resident):
    _, graphs, loaded = resident
    srv = im.Server(0, slots=3)
    try:
        for G in loaded:
            srv.add_graph(G)
        qs = [dict(graph=0, K=6, J=64, model={"kind": "wc"}, seed=11, rebuild_eps=0.01),
              dict(graph=2, K=4, J=16, model={"kind": "uniform", "p": 0.1}, seed=12, rebuild_eps=0.01),
              dict(graph=0, K=5, J=32, model={"kind": "trivalency", "seed": 5}, seed=13, rebuild_eps=-1.0)]
        tickets = [srv.submit(**q) for q in qs]
        res = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for q, r in zip(qs, res):
        g = graphs[q["graph"]]
        ref = O.select_seeds(g, O.thresholds(g, q["model"]), q["J"], q["K"], q["seed"], q["rebuild_eps"],
                             "reverse")
        assert r["seeds"].tolist() == list(ref["seeds"])


def test_admission_respects_budget(im, resident):
    _, graphs, loaded = resident
    qs = _queries(len(loaded), 10, seed=2)
    solo = [_solo(im, loaded, q) for q in qs]
    probe = im.Server(0, slots=1)
    try:
        for G in loaded:
            probe.add_graph(G)
        need = [probe.query_bytes(q["graph"], q["J"], q["K"]) for q in qs]
        graph_bytes = probe.stats()["graph_bytes"]
    finally:
        probe.close()
    budget = graph_bytes + int(1.5 * max(need))  # room for the largest query, not two of them
    srv = im.Server(0, slots=8, hbm_budget_bytes=budget, max_bypass=2)
    try:
        for G in loaded:
            srv.add_graph(G)
        tickets = [srv.submit(**q) for q in qs]
        res = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for r, s, b in zip(res, solo, need):
        assert r["status"] == 0, r["error"]
        assert r["bytes"] == b
        _same(r, s)
    assert st["reserved_peak"] <= budget - graph_bytes
    assert st["graph_bytes"] == graph_bytes


def test_query_larger_than_budget_is_refused(im, resident):
    _, graphs, loaded = resident
    probe = im.Server(0, slots=1)
    try:
        probe.add_graph(loaded[1])
        small = probe.query_bytes(0, 16, 1)
        big = probe.query_bytes(0, 1024, 5)
        graph_bytes = probe.stats()["graph_bytes"]
    finally:
        probe.close()
    assert big > 2 * small
    srv = im.Server(0, slots=2, hbm_budget_bytes=graph_bytes + small + small // 2)
    try:
        srv.add_graph(loaded[1])
        with pytest.raises(im.IMError) as e:
            srv.submit(graph=0, K=5, J=1024)
        assert e.value.status == -3
        r = srv.wait(srv.submit(graph=0, K=1, J=16, seed=4))
        assert r["status"] == 0 and r["bytes"] == small
        _same(r, im.im_select_seeds(loaded[1], 1, 16, seed=4, rebuild_eps=0.01))
    finally:
        srv.close()


def test_query_bytes_bounds_the_allocation(im, resident):
    # the worker's own context gets exactly query_bytes as its budget, so a
    # query that allocated more would fail with IM_E_NOMEM
    _, graphs, loaded = resident
    for gi, J, K in [(1, 1024, 50), (3, 64, 5), (2, 16, 1)]:
        probe = im.Server(0, slots=1)
        try:
            for G in loaded:
                probe.add_graph(G)
            need = probe.query_bytes(gi, J, K)
            graph_bytes = probe.stats()["graph_bytes"]
        finally:
            probe.close()
        srv = im.Server(0, slots=1, hbm_budget_bytes=graph_bytes + need)
        try:
            for G in loaded:
                srv.add_graph(G)
            r = srv.wait(srv.submit(graph=gi, K=K, J=J, seed=3))
        finally:
            srv.close()
        assert r["status"] == 0, r["error"]
        _same(r, im.im_select_seeds(loaded[gi], K, J, seed=3, rebuild_eps=0.01))


def test_submit_errors(im, resident):
    _, graphs, loaded = resident
    srv = im.Server(0, slots=2)
    try:
        srv.add_graph(loaded[0])
        for kw, status in [(dict(graph=5, K=1, J=64), -2), (dict(graph=0, K=graphs[0].n + 1, J=64), -2),
                           (dict(graph=0, K=1, J=48), -1),
                           (dict(graph=0, K=1, J=64, model={"kind": "uniform", "p": 1.5}), -1)]:
            with pytest.raises(im.IMError) as e:
                srv.submit(**kw)
            assert e.value.status == status, kw
        with pytest.raises(im.IMError) as e:
            srv.wait(12345)
        assert e.value.status == -2
        t = srv.submit(graph=0, K=3, J=64)  # the graph's own model (weighted cascade)
        r = srv.wait(t)
        assert r["status"] == 0
        _same(r, im.im_select_seeds(loaded[0], 3, 64, seed=2410, rebuild_eps=0.01))
    finally:
        srv.close()
