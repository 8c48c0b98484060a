"""Seeded synthetic workloads (graphs and per-edge weights).

This module generates inputs only; it holds none of the method's arithmetic
(no edge hashes, thresholds, sketches or simulations).  It is the one module
that both the oracle tests and the CUDA path consume.  The graphs stand in
for the SNAP social networks of the paper's evaluation (Sec. 5, Table 2):
R-MAT graphs are power-law like all seven of them, at the vertex scale of
Pokec / LiveJournal (scale 20) and Sinaweibo (scale 24).

The C source (``gen.c``) is compiled on first use into ``_libworkloads.so``
next to it (``build()`` does it explicitly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "_libworkloads.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (gcc, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.wl_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.wl_rmat.restype = ctypes.c_int64
        lib.wl_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
        lib.wl_erdos_renyi.restype = ctypes.c_int64
        lib.wl_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, i32p, i32p, ctypes.c_int64]
        lib.wl_chung_lu.restype = ctypes.c_int64
        lib.wl_edge_weights.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_float)]
        lib.wl_edge_weights.restype = None
        lib.wl_splitmix_outputs.argtypes = [ctypes.c_uint64, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_uint64)]
        lib.wl_splitmix_outputs.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class Graph:
    """CSR of out-edges: rowptr[n+1], col[m] (int32, rows sorted, no dups/loops)."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def indegree(self) -> np.ndarray:
        return np.bincount(self.col, minlength=self.n).astype(np.int64)


def from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR from an explicit (u, v) edge list (small hand-made test graphs)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    if e.size:
        order = np.lexsort((e[:, 1], e[:, 0]))
        e = e[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, e[:, 0] + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return Graph(n, rowptr, e[:, 1].astype(np.int32).copy(), name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2410) -> Graph:
    lib = _load()
    n = 1 << scale
    draws = edge_factor * n
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col = np.empty(max(draws, 1), dtype=np.int32)
    m = lib.wl_rmat(scale, draws, a, b, c, seed & (2**64 - 1), _ptr(rowptr, ctypes.c_int32),
                    _ptr(col, ctypes.c_int32))
    if m < 0:
        raise RuntimeError(f"wl_rmat failed ({m})")
    return Graph(n, rowptr, col[:m].copy(), f"rmat{scale}_ef{edge_factor}")


def erdos_renyi(n: int, m: int, seed: int = 2410) -> Graph:
    lib = _load()
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col = np.empty(max(m, 1), dtype=np.int32)
    got = lib.wl_erdos_renyi(n, m, seed & (2**64 - 1), _ptr(rowptr, ctypes.c_int32),
                             _ptr(col, ctypes.c_int32))
    if got != m:
        raise RuntimeError(f"wl_erdos_renyi failed ({got})")
    return Graph(n, rowptr, col[:m].copy(), f"er{n}_{m}")


def chung_lu(n: int, avg_deg: float, gamma: float = 2.1, seed: int = 2410) -> Graph:
    lib = _load()
    cap = int(n * avg_deg * 1.5) + 1024
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col = np.empty(cap, dtype=np.int32)
    m = lib.wl_chung_lu(n, float(avg_deg), float(gamma), seed & (2**64 - 1),
                        _ptr(rowptr, ctypes.c_int32), _ptr(col, ctypes.c_int32), cap)
    if m < 0:
        raise RuntimeError(f"wl_chung_lu failed ({m})")
    return Graph(n, rowptr, col[:m].copy(), f"cl{n}_{avg_deg:g}")


def edge_weights(m: int, kind: str, p0: float, p1: float, seed: int = 2410) -> np.ndarray:
    """Per-edge probabilities: kind 'normal' -> N(p0, p1) clipped to [0,1], 'uniform' -> U(p0, p1)."""
    lib = _load()
    w = np.empty(max(m, 1), dtype=np.float32)
    lib.wl_edge_weights(m, 0 if kind == "normal" else 1, p0, p1, seed & (2**64 - 1),
                        _ptr(w, ctypes.c_float))
    return w[:m].copy()


def splitmix_outputs(seed: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.wl_splitmix_outputs(seed & (2**64 - 1), count, _ptr(out, ctypes.c_uint64))
    return out


# ---------------------------------------------------------------------------
# Named workloads (the paper's workload shapes, synthetic stand-ins)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    graph_fn: object
    model: dict
    J: int
    K: int
    seed: int = 2410
    rebuild_eps: float = 0.01
    notes: str = ""
    _graph: Graph | None = field(default=None, repr=False)

    def graph(self) -> Graph:
        if self._graph is None:
            self._graph = self.graph_fn()
        return self._graph


def workload(name: str) -> Workload:
    """The plain-method workloads: er10k (tiny), rmat20 (mid), rmat24 (large);
    rmat22 is the large workload's shape at a quarter of its size (profiling
    captures that must stay within a few GB of device memory)."""
    if name == "er10k":
        return Workload("er10k: ER n=10000 m=100000, IC p=0.01, J=64, K=10",
                        lambda: erdos_renyi(10_000, 100_000, seed=2410),
                        {"kind": "uniform", "p": 0.01}, J=64, K=10)
    if name == "rmat20":
        return Workload("rmat20: R-MAT scale 20 ef 16 (0.57/0.19/0.19), WC, J=256, K=50",
                        lambda: rmat(20, 16, seed=2410), {"kind": "wc"}, J=256, K=50)
    if name == "rmat24":
        return Workload("rmat24: R-MAT scale 24 ef 16 (0.57/0.19/0.19), trivalency, J=512, K=50",
                        lambda: rmat(24, 16, seed=2410), {"kind": "trivalency", "seed": 2410},
                        J=512, K=50)
    if name == "rmat22":
        return Workload("rmat22: R-MAT scale 22 ef 16 (0.57/0.19/0.19), trivalency, J=512, K=50",
                        lambda: rmat(22, 16, seed=2410), {"kind": "trivalency", "seed": 2410},
                        J=512, K=50)
    raise KeyError(name)


def batched_workload(G: int = 512, seed: int = 2410):
    """The batched form: G directed Chung-Lu graphs (gamma 2.1), n uniform in
    [1000, 200000], average degree uniform in [8, 32]; per graph K uniform in
    [5, 50], J in {64, 128}, uniform IC p in [0.005, 0.05].  Returns
    (graphs, p, J, K)."""
    rng = np.random.default_rng(seed)
    graphs, p, J, K = [], [], [], []
    for i in range(G):
        n = int(rng.integers(1000, 200001))
        d = float(rng.uniform(8, 32))
        graphs.append(chung_lu(n, d, 2.1, seed=seed * 1000 + i))
        p.append(float(np.float32(rng.uniform(0.005, 0.05))))
        J.append(int(rng.choice([64, 128])))
        K.append(int(rng.integers(5, 51)))
    return graphs, p, J, K


# Served form: 16 resident R-MAT graphs (edge factor 16), scales 14..22 spread
# evenly with the lower scales repeated.
SERVED_SCALES = (14, 15, 16, 17, 18, 19, 20, 21, 22, 14, 15, 16, 17, 18, 19, 20)


def served_graphs(seed: int = 2410, scales=SERVED_SCALES) -> list:
    return [rmat(s, 16, seed=seed + 17 * i) for i, s in enumerate(scales)]


def served_queries(count: int, rate: float = 200.0, n_graphs: int = len(SERVED_SCALES),
                   seed: int = 2410) -> list:
    """Poisson arrivals (mean `rate` per second, first at t = 0) of queries:
    graph uniform over the resident graphs, K in {10, 25, 50}, J in
    {64, 256, 1024}, model uniform p = 0.01 or weighted cascade, rebuild
    threshold 0.01, simulation seed drawn per query."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    gaps[0] = 0.0
    arrival = np.cumsum(gaps)
    out = []
    for i in range(count):
        model = {"kind": "uniform", "p": 0.01} if rng.integers(2) == 0 else {"kind": "wc"}
        out.append({"arrival_s": float(arrival[i]), "graph": int(rng.integers(n_graphs)),
                    "K": int(rng.choice([10, 25, 50])), "J": int(rng.choice([64, 256, 1024])),
                    "model": model, "seed": int(rng.integers(1 << 40)), "rebuild_eps": 0.01})
    return out
