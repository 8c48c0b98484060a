"""ORACLE — plain CPU implementation of DiFuseR's sketch-based IM (arXiv 2410.14047).

Test infrastructure only.  It shares no code with the CUDA library and must
only be imported by the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.

The arithmetic lives in ``oracle.c`` (compiled with gcc + OpenMP into
``_liboracle.so`` next to it); this module only marshals numpy arrays.
``mc.py`` holds the independent Monte-Carlo spread oracle that uses a
standard RNG instead of hash sampling (Sec. 5.1).

Function-level citations are in ``oracle.c``.  Parity unpinned: none of the
functions here is unpinned; see the test suite for the pin of each one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

MODEL_KINDS = {"uniform": 0, "wc": 1, "trivalency": 2, "explicit": 3, "target": 4}
PHI = 0.77351
VISITED = 0xFF


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB_PATH)
    u8, i32, u32, u64, f32, f64 = (ctypes.c_uint8, ctypes.c_int32, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_float, ctypes.c_double)
    P = ctypes.POINTER
    i64 = ctypes.c_int64
    sig = {
        "orc_murmur3_32": (u32, [P(u8), i64, u32]),
        "orc_edge_hash": (u32, [i32, i32]),
        "orc_rank": (i32, [i32, u32]),
        "orc_splitmix64": (u64, [P(u64)]),
        "orc_draw_sims": (None, [u64, i32, P(u32), P(u32)]),
        "orc_prob_threshold": (u32, [f32]),
        "orc_thresholds": (ctypes.c_int, [i32, i64, P(i32), P(i32), i32, f32, u64, P(f32), P(u32)]),
        "orc_fill": (None, [i32, i32, P(u32), P(u8)]),
        "orc_build_bruteforce": (None, [i32, i64, P(i32), P(i32), P(u32), i32, P(u32), P(u32), P(u8)]),
        "orc_build_jacobi": (i32, [i32, i64, P(i32), P(i32), P(u32), i32, P(u32), P(u32), P(u8)]),
        "orc_build_reverse": (None, [i32, i64, P(i32), P(i32), P(u32), i32, P(u32), P(u32), P(u8)]),
        "orc_sums": (None, [i32, i32, P(u8), P(u64)]),
        "orc_pick": (i32, [i32, P(u64), P(u8)]),
        "orc_estimate": (f64, [i32, u64]),
        "orc_cover": (u64, [i32, i64, P(i32), P(i32), P(u32), i32, P(u32), P(u8), i32]),
        "orc_count_visited": (u64, [i64, P(u8)]),
        "orc_rebuild_due": (ctypes.c_int, [u64, u64, i32, f64]),
        "orc_select_seeds": (ctypes.c_int, [i32, i64, P(i32), P(i32), P(u32), i32, i32, u64, f64,
                                            i32, P(i32), P(f64), P(f64), P(u8), P(i32)]),
        "orc_spread_hash": (None, [i32, i64, P(i32), P(i32), P(u32), P(i32), i32, i64, u64,
                                   P(u64), P(u64)]),
        "orc_spread_ic": (None, [i32, i64, P(i32), P(i32), P(u32), P(i32), i32, i64, u64,
                                 P(u64), P(u64)]),
        "orc_register_entry": (i32, [i32, i64, P(i32), P(i32), P(u32), u32, u32, ctypes.c_void_p,
                                     i32]),
        "orc_reach_mark": (i64, [i32, i64, P(i32), P(i32), P(u32), u32, P(i32), i32, P(u8)]),
        "orc_num_threads": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _u64(x: int) -> int:
    return int(x) & (2**64 - 1)


# --- primitives -------------------------------------------------------------

def murmur3_32(data: bytes, seed: int = 0) -> int:
    L = _load()
    buf = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)
    return int(L.orc_murmur3_32(_p(buf, ctypes.c_uint8), len(data), seed & 0xFFFFFFFF))


def edge_hash(u: int, v: int) -> int:
    return int(_load().orc_edge_hash(u, v))


def rank(u: int, salt: int) -> int:
    return int(_load().orc_rank(u, salt & 0xFFFFFFFF))


def splitmix64(seed: int, count: int) -> np.ndarray:
    L = _load()
    st = ctypes.c_uint64(_u64(seed))
    return np.array([L.orc_splitmix64(ctypes.byref(st)) for _ in range(count)], dtype=np.uint64)


def draw_sims(seed: int, J: int):
    """Sorted (X, salt) pairs of the J simulations (Sec. 2.2, Sec. 4.1)."""
    L = _load()
    X = np.empty(J, dtype=np.uint32)
    salt = np.empty(J, dtype=np.uint32)
    L.orc_draw_sims(_u64(seed), J, _p(X, ctypes.c_uint32), _p(salt, ctypes.c_uint32))
    return X, salt


def prob_threshold(w: float) -> int:
    return int(_load().orc_prob_threshold(float(np.float32(w))))


def thresholds(g, model: dict) -> np.ndarray:
    """Per-out-edge uint32 thresholds of a diffusion model (Sec. 2.1)."""
    L = _load()
    kind = MODEL_KINDS[model["kind"]]
    thr = np.empty(max(g.m, 1), dtype=np.uint32)
    w = np.ascontiguousarray(model.get("w", np.zeros(1, np.float32)), dtype=np.float32)
    rc = L.orc_thresholds(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32), kind,
                          float(model.get("p", 0.0)), _u64(model.get("seed", 0)),
                          _p(w, ctypes.c_float), _p(thr, ctypes.c_uint32))
    if rc != 0:
        raise ValueError(model)
    return thr[: g.m]


# --- build ----------------------------------------------------------------------

def _build(fn, g, thr, J, X, salt, M):
    L = _load()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    return getattr(L, fn)(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                          _p(thr, ctypes.c_uint32), J, _p(X, ctypes.c_uint32),
                          _p(salt, ctypes.c_uint32), _p(M, ctypes.c_uint8))


def empty_registers(n: int, J: int) -> np.ndarray:
    return np.zeros((n, J), dtype=np.uint8)


def fill(g, J, salt, M):
    _load().orc_fill(g.n, J, _p(salt, ctypes.c_uint32), _p(M, ctypes.c_uint8))
    return M


def build_bruteforce(g, thr, J, X, salt, M=None):
    M = empty_registers(g.n, J) if M is None else M
    _build("orc_build_bruteforce", g, thr, J, X, salt, M)
    return M


def build_jacobi(g, thr, J, X, salt, M=None):
    M = empty_registers(g.n, J) if M is None else M
    sweeps = _build("orc_build_jacobi", g, thr, J, X, salt, M)
    return M, int(sweeps)


def build_reverse(g, thr, J, X, salt, M=None):
    M = empty_registers(g.n, J) if M is None else M
    _build("orc_build_reverse", g, thr, J, X, salt, M)
    return M


# --- estimate / pick / cover ---------------------------------------------------

def sums(M: np.ndarray) -> np.ndarray:
    n, J = M.shape
    S = np.empty(max(n, 1), dtype=np.uint64)
    _load().orc_sums(n, J, _p(np.ascontiguousarray(M), ctypes.c_uint8), _p(S, ctypes.c_uint64))
    return S[:n]


def pick(S: np.ndarray, is_seed: np.ndarray) -> int:
    S = np.ascontiguousarray(S, dtype=np.uint64)
    is_seed = np.ascontiguousarray(is_seed, dtype=np.uint8)
    return int(_load().orc_pick(S.shape[0], _p(S, ctypes.c_uint64), _p(is_seed, ctypes.c_uint8)))


def estimate(J: int, S: int) -> float:
    return float(_load().orc_estimate(J, int(S)))


def cover(g, thr, J, X, M, s) -> int:
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    return int(_load().orc_cover(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                                 _p(thr, ctypes.c_uint32), J, _p(X, ctypes.c_uint32),
                                 _p(M, ctypes.c_uint8), int(s)))


def count_visited(M) -> int:
    return int(_load().orc_count_visited(M.size, _p(np.ascontiguousarray(M), ctypes.c_uint8)))


def rebuild_due(count: int, oldcount: int, J: int, eps: float) -> bool:
    return bool(_load().orc_rebuild_due(count, oldcount, J, eps))


BUILD_MODES = {"jacobi": 0, "reverse": 1, "bruteforce": 2}


def select_seeds(g, thr, J: int, K: int, seed: int, eps: float = 0.01, build: str = "reverse"):
    """Alg. 4 on one device.  Returns dict(seeds, score, est, M, rebuilds)."""
    L = _load()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    seeds = np.empty(max(K, 1), dtype=np.int32)
    score = np.empty(max(K, 1), dtype=np.float64)
    est = np.empty(max(K, 1), dtype=np.float64)
    M = np.empty((g.n, J), dtype=np.uint8)
    reb = ctypes.c_int32(0)
    rc = L.orc_select_seeds(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                            _p(thr, ctypes.c_uint32), J, K, _u64(seed), float(eps),
                            BUILD_MODES[build], _p(seeds, ctypes.c_int32), _p(score, ctypes.c_double),
                            _p(est, ctypes.c_double), _p(M, ctypes.c_uint8), ctypes.byref(reb))
    if rc != 0:
        raise ValueError("K > n")
    return {"seeds": seeds[:K].copy(), "score": score[:K].copy(), "est": est[:K].copy(), "M": M,
            "rebuilds": int(reb.value)}


def _spread(fn, g, thr, seeds, R, seed):
    L = _load()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
    getattr(L, fn)(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                      _p(thr, ctypes.c_uint32), _p(s, ctypes.c_int32), s.shape[0], int(R),
                      _u64(seed), ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


def spread_hash(g, thr, seeds, R: int, seed: int):
    """Hash-sampled spread over R fused-sampling simulations: (sum |reach|, sum |reach|^2)."""
    return _spread("orc_spread_hash", g, thr, seeds, R, seed)


def spread_ic(g, thr, seeds, R: int, seed: int):
    """IC Monte-Carlo spread with independent counter-based coins: (sum, sum of squares)."""
    return _spread("orc_spread_ic", g, thr, seeds, R, seed)


def register_entry(g, thr, Xj: int, saltj: int, u: int, vis=None) -> int:
    """One register by BFS: max rank over R*_j(u) (vis: n bytes, nonzero = visited)."""
    L = _load()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    vp = None if vis is None else np.ascontiguousarray(vis, dtype=np.uint8).ctypes.data_as(ctypes.c_void_p)
    return int(L.orc_register_entry(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                                    _p(thr, ctypes.c_uint32), int(Xj), int(saltj), vp, int(u)))


def reach_mark(g, thr, Xj: int, seeds) -> np.ndarray:
    """Boolean reach set of a seed set in one simulation."""
    L = _load()
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    if thr.size == 0:
        thr = np.zeros(1, np.uint32)
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    mark = np.empty(max(g.n, 1), dtype=np.uint8)
    L.orc_reach_mark(g.n, g.m, _p(g.rowptr, ctypes.c_int32), _p(g.col, ctypes.c_int32),
                     _p(thr, ctypes.c_uint32), int(Xj), _p(s, ctypes.c_int32), s.shape[0],
                     _p(mark, ctypes.c_uint8))
    return mark[: g.n].astype(bool)


def num_threads() -> int:
    return int(_load().orc_num_threads())
