"""The seeded input generators produce canonical CSR graphs of the stated shapes."""
import numpy as np

import workloads as W


def _check_csr(g):
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.m
    assert (np.diff(g.rowptr) >= 0).all()
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    assert (g.col >= 0).all() and (g.col < g.n).all()
    assert (src != g.col).all()  # no self-loops
    key = src.astype(np.int64) * g.n + g.col
    assert (np.diff(key) > 0).all()  # rows sorted, no duplicates


def test_erdos_renyi_exact_m():
    g = W.erdos_renyi(10_000, 100_000, seed=2410)
    assert g.m == 100_000
    _check_csr(g)


def test_rmat_shape_and_determinism():
    g = W.rmat(14, 16, seed=5)
    _check_csr(g)
    g2 = W.rmat(14, 16, seed=5)
    assert (g.col == g2.col).all() and (g.rowptr == g2.rowptr).all()
    deg = np.diff(g.rowptr)
    # power-law skew: vertex 0 is the biggest hub, many vertices are empty
    assert deg[0] == deg.max() and deg.max() > 50 * deg.mean()
    assert (deg == 0).sum() > 0.1 * g.n


def test_chung_lu_shape():
    g = W.chung_lu(20_000, 12.0, 2.1, seed=3)
    _check_csr(g)
    assert 0.7 * 12 * g.n < g.m < 1.1 * 12 * g.n
    deg = np.diff(g.rowptr)
    assert deg[:10].mean() > 20 * deg.mean()


def test_edge_weights_ranges():
    w = W.edge_weights(100_000, "normal", 0.05, 0.025, seed=1)
    assert w.min() >= 0 and w.max() <= 1 and abs(w.mean() - 0.05) < 0.002
    u = W.edge_weights(100_000, "uniform", 0.0, 0.1, seed=1)
    assert u.min() >= 0 and u.max() < 0.1 and abs(u.mean() - 0.05) < 0.001
