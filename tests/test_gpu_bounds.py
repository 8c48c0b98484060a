"""The bounds-checked variant of the library on the small parity cases.

_libdifuser_im_bounds.so is the same sources compiled with IM_BOUNDS_CHECK:
every checked device index (vertex ids read from edges, lists and queues, edge
and list offsets, bucket ids, chunk numbers) is tested against its range, and a
bad one raises an error bit that the call returns as IM_E_STATE, with the
access redirected to a valid address instead of faulting.  It stands in for a
memory checker: every schedule of the hot path (edge scans and bucketed lists,
one cooperative launch per phase and one launch per level, full and incremental
rebuilds) runs here on small graphs, and each must finish without a raised
bit and with the oracle's seeds, scores and registers.
"""
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
    from paper_2410_14047_gb300 import _build
    _build.build_bounds()
    lib.load_library(lib.BOUNDS_LIB_PATH)
    return lib


GRAPHS = {
    "er2k": lambda: W.erdos_renyi(2000, 16000, seed=3),
    "rmat11": lambda: W.rmat(11, 16, seed=5),
    "cl3k": lambda: W.chung_lu(3000, 12.0, 2.1, seed=9),
    "path": lambda: W.from_edges(60, [(i, i + 1) for i in range(59)]),
    "star_in": lambda: W.from_edges(300, [(i, 0) for i in range(1, 300)]),
}
MODELS = {"p30": {"kind": "uniform", "p": 0.3}, "wc": {"kind": "wc"},
          "tri": {"kind": "trivalency", "seed": 2410}, "p1": {"kind": "uniform", "p": 1.0}}
SCHEDULES = {
    "buckets": {},
    "scans": {"buckets": 0, "incremental": 2, "heavy_indeg": 8},
    "levels": {"persistent": 0, "dense_div": 2},
    "full_rebuilds": {"incremental": 0, "chain": 0, "lazy_pick": 0},
    "dense_walks": {"buckets": 0, "dense_div": 1000000, "dense_out": 1, "incremental": 0},
    "dense_all_sims": {"buckets": 0, "dense_div": 1000000, "dense_out": 1, "dense_all": 3, "incremental": 2},
}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("gname,mname", [("er2k", "p30"), ("rmat11", "wc"), ("cl3k", "tri"), ("path", "p1"),
                                         ("star_in", "wc")])
def test_bounds_checked_selection_matches_oracle(im, sched, gname, mname):
    g = GRAPHS[gname]()
    model = MODELS[mname]
    ctx = im.im_ctx_create(0, lib_path=im.BOUNDS_LIB_PATH)
    im.im_ctx_set_tuning(ctx, SCHEDULES[sched])
    G = im.im_graph_load(ctx, g.rowptr, g.col, model)
    J, K, seed = 64, 6, 17
    r = im.im_select_seeds(G, K, J, seed=seed, return_sketch=True)
    ref = O.select_seeds(g, O.thresholds(g, model), J, K, seed, 0.01, "reverse")
    assert r["seeds"].tolist() == ref["seeds"].tolist()
    assert np.array_equal(r["score"], ref["score"])
    assert np.array_equal(r["sketch"].registers(), ref["M"])


def test_bounds_checked_build_at_every_J(im):
    g = W.rmat(10, 16, seed=8)
    model = {"kind": "wc"}
    ctx = im.im_ctx_create(0, lib_path=im.BOUNDS_LIB_PATH)
    G = im.im_graph_load(ctx, g.rowptr, g.col, model)
    thr = O.thresholds(g, model)
    for J in (16, 32, 128, 512, 1024):
        sk = im.im_sketch_build(G, J, J + 1)
        X, salt = O.draw_sims(J + 1, J)
        assert np.array_equal(sk.registers(), O.build_reverse(g, thr, J, X, salt)), J
