"""Python binding of the DiFuseR GB300 library (C ABI in include/difuser_im.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``_libdifuser_im.so``.  Functions carry the C names.  PyTorch is
used for device memory (the library allocates through torch's caching
allocator when torch has CUDA) and for the current CUDA stream.

There is no CPU fallback: when the compiled library is missing, every call
raises ``IMError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_libdifuser_im.so")
# the bounds-checked test variant of the same sources (see _build.py)
BOUNDS_LIB_PATH = os.path.join(HERE, "_libdifuser_im_bounds.so")

MODEL_KINDS = {"uniform": 0, "wc": 1, "trivalency": 2, "explicit": 3, "target": 4}
STATUS = {0: "IM_OK", -1: "IM_E_INVAL", -2: "IM_E_RANGE", -3: "IM_E_NOMEM", -4: "IM_E_CUDA",
          -5: "IM_E_TIMEOUT", -6: "IM_E_STATE"}

# Every symbol the C header declares, for the load check.
EXPORTS = ["im_ctx_create", "im_ctx_destroy", "im_ctx_bytes_in_use", "im_ctx_bytes_peak",
           "im_last_error", "im_status_str", "im_last_stats", "im_ctx_set_timing",
           "im_ctx_set_trace", "im_last_trace", "im_ctx_set_tuning", "im_ctx_get_tuning",
           "im_ctx_set_limits",
           "im_graph_load", "im_graph_free",
           "im_graph_info", "im_sketch_build", "im_sketch_free", "im_sketch_registers",
           "im_sketch_set_registers", "im_sketch_sims", "im_sketch_sums", "im_sketch_pick",
           "im_sketch_cover", "im_sketch_rebuild", "im_select_seeds", "im_spread_mc",
           "im_argmax_noalloc", "im_batch_load", "im_batch_free", "im_batch_select_seeds",
           "im_server_create", "im_server_destroy", "im_server_add_graph", "im_server_query_bytes",
           "im_server_submit", "im_server_wait", "im_server_get_stats", "im_server_clock_ms",
           "im_fill_rate"]


class IMError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class im_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("w", ctypes.POINTER(ctypes.c_float))]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class im_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


class im_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("ms_total", "ms_build", "ms_rebuild", "ms_pick",
                                               "ms_propagate", "ms_cover_kernels",
                                               "ms_pick_kernels", "ms_fill_kernels")] + \
               [(k, ctypes.c_int64) for k in ("launches", "sweep_launches", "builds", "sweeps",
                                              "cover_levels")] + \
               [(k, ctypes.c_uint64) for k in ("sweep_vertices", "sweep_edges", "sweep_chunks",
                                               "sweep_cas", "sweep_changed", "cover_edges",
                                               "cover_chunks", "visited", "alg_bytes_sweep",
                                               "sweep_heavy", "sweep_heavy_sims", "sweep_batches",
                                               "sweep_dealt", "sweep_edges_live", "sweep_buckets",
                                               "sweep_bucket_entries", "affected",
                                               "pull_buckets", "pull_entries",
                                               "sweep_changed_buckets", "pick_refreshed")]


class im_tuning(ctypes.Structure):
    _fields_ = [("heavy_indeg", ctypes.c_int32), ("light_batches", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("dense_div", ctypes.c_int32),
                ("lazy_pick", ctypes.c_int32), ("buckets", ctypes.c_int32), ("incremental", ctypes.c_int32),
                ("chain", ctypes.c_int32), ("pick_tile", ctypes.c_int32), ("dense_out", ctypes.c_int32),
                ("dense_all", ctypes.c_int32)]


class im_trace_rec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("count", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("ms", ctypes.c_double)]


class im_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("max_bypass", ctypes.c_int32)]


class im_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("K", ctypes.c_int32), ("J", ctypes.c_int32),
                ("model", im_model), ("seed", ctypes.c_uint64), ("rebuild_eps", ctypes.c_double)]


class im_query_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("ms_select", ctypes.c_double),
                ("bytes", ctypes.c_uint64), ("error", ctypes.c_char * 160)]


class im_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "bypassed")] + \
               [(k, ctypes.c_int32) for k in ("slots", "running", "running_peak", "pending")] + \
               [(k, ctypes.c_uint64) for k in ("budget", "graph_bytes", "reserved", "reserved_peak")]


_libs = {}


def load_library(path: str = LIB_PATH):
    """Load the compiled library and declare the C signatures."""
    path = os.path.abspath(path)
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise IMError(-4, f"CUDA library not built ({path}); run paper_2410_14047_gb300._build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "im_ctx_create": (ctypes.c_int, [ctypes.c_int, vp, u64, P(im_allocator), P(vp)]),
        "im_ctx_destroy": (None, [vp]),
        "im_ctx_bytes_in_use": (u64, [vp]),
        "im_ctx_bytes_peak": (u64, [vp]),
        "im_last_error": (ctypes.c_char_p, [vp]),
        "im_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "im_last_stats": (ctypes.c_int, [vp, P(im_stats)]),
        "im_ctx_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "im_ctx_set_trace": (ctypes.c_int, [vp, ctypes.c_int]),
        "im_last_trace": (i64, [vp, P(im_trace_rec), i64]),
        "im_ctx_set_tuning": (ctypes.c_int, [vp, P(im_tuning)]),
        "im_ctx_get_tuning": (ctypes.c_int, [vp, P(im_tuning)]),
        "im_ctx_set_limits": (ctypes.c_int, [vp, u64, i32]),
        "im_graph_load": (ctypes.c_int, [vp, i32, i64, P(i32), P(i32), P(im_model), P(vp)]),
        "im_graph_free": (None, [vp]),
        "im_graph_info": (ctypes.c_int, [vp, P(i32), P(i64)]),
        "im_sketch_build": (ctypes.c_int, [vp, i32, u64, P(vp)]),
        "im_sketch_free": (None, [vp]),
        "im_sketch_registers": (ctypes.c_int, [vp, P(ctypes.c_uint8)]),
        "im_sketch_set_registers": (ctypes.c_int, [vp, P(ctypes.c_uint8)]),
        "im_sketch_sims": (ctypes.c_int, [vp, P(ctypes.c_uint32), P(ctypes.c_uint32)]),
        "im_sketch_sums": (ctypes.c_int, [vp, P(u64)]),
        "im_sketch_pick": (ctypes.c_int, [vp, P(i32), P(u64), P(f64)]),
        "im_sketch_cover": (ctypes.c_int, [vp, i32, P(u64)]),
        "im_sketch_rebuild": (ctypes.c_int, [vp]),
        "im_select_seeds": (ctypes.c_int, [vp, i32, i32, P(im_model), u64, f64, P(i32), P(f64),
                                           P(f64), P(vp)]),
        "im_spread_mc": (ctypes.c_int, [vp, P(i32), i32, i64, u64, P(f64), P(f64), P(u64), P(u64)]),
        "im_argmax_noalloc": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "im_batch_load": (ctypes.c_int, [vp, i32, P(i32), P(i64), P(P(i32)), P(P(i32)), P(ctypes.c_float),
                                         P(vp)]),
        "im_batch_free": (None, [vp]),
        "im_batch_select_seeds": (ctypes.c_int, [vp, P(i32), P(i32), u64, f64, P(i32), P(f64), P(f64)]),
        "im_server_create": (ctypes.c_int, [P(im_server_config), P(vp)]),
        "im_server_destroy": (None, [vp]),
        "im_server_add_graph": (ctypes.c_int, [vp, vp, P(i32)]),
        "im_server_query_bytes": (ctypes.c_int, [vp, i32, i32, i32, P(u64)]),
        "im_server_submit": (ctypes.c_int, [vp, P(im_query), P(i32), P(f64), P(f64), P(i64)]),
        "im_server_wait": (ctypes.c_int, [vp, i64, f64, P(im_query_result)]),
        "im_server_get_stats": (ctypes.c_int, [vp, P(im_server_stats)]),
        "im_server_clock_ms": (f64, []),
        "im_fill_rate": (ctypes.c_int, [vp, i32, u64, P(im_model), P(u64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _libs[path] = L
    return L


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _u64(x: int) -> int:
    return int(x) & (2**64 - 1)


def _model(model: dict | None, keep: list):
    if model is None:
        return None
    m = im_model()
    m.kind = MODEL_KINDS[model["kind"]]
    m.p = float(model.get("p", 0.0))
    m.seed = _u64(model.get("seed", 0))
    if model["kind"] in ("explicit", "target"):
        w = np.ascontiguousarray(model["w"], dtype=np.float32)
        keep.append(w)
        m.w = _p(w, ctypes.c_float)
    return m


class _TorchAllocator:
    """Device memory from torch's caching allocator, handed to the C library."""

    def __init__(self, device: int):
        import torch

        def alloc(nbytes, stream, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
            except Exception:  # out of memory: the library reports IM_E_NOMEM
                return None

        def free(ptr, nbytes, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = _ALLOC_FN(alloc)
        self._free = _FREE_FN(free)
        self.struct = im_allocator(self._alloc, self._free, None)


class Context:
    def __init__(self, handle, lib, allocator, device, stream):
        self.handle = handle
        self.lib = lib
        self._allocator = allocator
        self.device = device
        self.stream = stream

    def check(self, st: int):
        if st != 0:
            raise IMError(st, self.lib.im_last_error(self.handle).decode(errors="replace"))

    def close(self):
        if self.handle:
            self.lib.im_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, ctx: Context, handle, n: int, m: int):
        self.ctx, self.handle, self.n, self.m = ctx, handle, n, m

    def free(self):
        if self.handle:
            self.ctx.lib.im_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Sketch:
    def __init__(self, graph: Graph, handle, J: int):
        self.graph, self.handle, self.J = graph, handle, J

    @property
    def _L(self):
        return self.graph.ctx.lib

    def _ck(self, st):
        self.graph.ctx.check(st)

    def registers(self) -> np.ndarray:
        out = np.empty((self.graph.n, self.J), dtype=np.uint8)
        self._ck(self._L.im_sketch_registers(self.handle, _p(out, ctypes.c_uint8)))
        return out

    def set_registers(self, M: np.ndarray):
        M = np.ascontiguousarray(M, dtype=np.uint8)
        assert M.shape == (self.graph.n, self.J)
        self._ck(self._L.im_sketch_set_registers(self.handle, _p(M, ctypes.c_uint8)))

    def sims(self):
        X = np.empty(self.J, dtype=np.uint32)
        s = np.empty(self.J, dtype=np.uint32)
        self._ck(self._L.im_sketch_sims(self.handle, _p(X, ctypes.c_uint32), _p(s, ctypes.c_uint32)))
        return X, s

    def sums(self) -> np.ndarray:
        out = np.empty(self.graph.n, dtype=np.uint64)
        self._ck(self._L.im_sketch_sums(self.handle, _p(out, ctypes.c_uint64)))
        return out

    def pick(self):
        s, S, e = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_double()
        self._ck(self._L.im_sketch_pick(self.handle, ctypes.byref(s), ctypes.byref(S), ctypes.byref(e)))
        return int(s.value), int(S.value), float(e.value)

    def cover(self, s: int) -> int:
        c = ctypes.c_uint64()
        self._ck(self._L.im_sketch_cover(self.handle, int(s), ctypes.byref(c)))
        return int(c.value)

    def rebuild(self):
        self._ck(self._L.im_sketch_rebuild(self.handle))

    def free(self):
        if self.handle:
            self._L.im_sketch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------

def im_ctx_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0,
                  torch_allocator: bool = True, lib_path: str = LIB_PATH) -> Context:
    L = load_library(lib_path)
    allocator = None
    if stream is None or torch_allocator:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        if torch_allocator:
            allocator = _TorchAllocator(device)
    h = ctypes.c_void_p()
    st = L.im_ctx_create(device, ctypes.c_void_p(int(stream) if stream else None), int(hbm_budget_bytes),
                         ctypes.byref(allocator.struct) if allocator else None, ctypes.byref(h))
    if st != 0:
        raise IMError(st, "im_ctx_create")
    return Context(h, L, allocator, device, stream)


def im_graph_load(ctx: Context, rowptr, col, model: dict) -> Graph:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = rowptr.shape[0] - 1
    m = col.shape[0]
    keep = []
    mdl = _model(model, keep)
    colp = col if m > 0 else np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.im_graph_load(ctx.handle, n, m, _p(rowptr, ctypes.c_int32),
                                    _p(colp, ctypes.c_int32), ctypes.byref(mdl), ctypes.byref(h)))
    return Graph(ctx, h, n, m)


def im_sketch_build(graph: Graph, J: int, seed: int) -> Sketch:
    h = ctypes.c_void_p()
    graph.ctx.check(graph.ctx.lib.im_sketch_build(graph.handle, int(J), _u64(seed), ctypes.byref(h)))
    return Sketch(graph, h, J)


def im_select_seeds(graph: Graph, K: int, J: int, model: dict | None = None, seed: int = 2410,
                    rebuild_eps: float = 0.01, return_sketch: bool = False) -> dict:
    keep = []
    mdl = _model(model, keep)
    seeds = np.empty(K, dtype=np.int32)
    score = np.empty(K, dtype=np.float64)
    est = np.empty(K, dtype=np.float64)
    h = ctypes.c_void_p()
    L = graph.ctx.lib
    graph.ctx.check(L.im_select_seeds(graph.handle, int(K), int(J),
                                      ctypes.byref(mdl) if mdl is not None else None, _u64(seed),
                                      float(rebuild_eps), _p(seeds, ctypes.c_int32),
                                      _p(score, ctypes.c_double), _p(est, ctypes.c_double),
                                      ctypes.byref(h) if return_sketch else None))
    out = {"seeds": seeds, "score": score, "est": est}
    if return_sketch:
        out["sketch"] = Sketch(graph, h, J)
    return out


def im_fill_rate(graph: Graph, J: int, seed: int = 2410, model: dict | None = None) -> dict:
    """Warp fill rate of the live tests, draw order vs sorted X (Table 6 analogue)."""
    keep = []
    mdl = _model(model, keep)
    out = np.zeros(5, dtype=np.uint64)
    graph.ctx.check(graph.ctx.lib.im_fill_rate(graph.handle, int(J), _u64(seed),
                                               ctypes.byref(mdl) if mdl is not None else None,
                                               _p(out, ctypes.c_uint64)))
    edges, live, wdraw, wsort, cands = (int(x) for x in out)
    return {"edges": edges, "live": live, "warps_draw": wdraw, "warps_sorted": wsort, "candidates": cands,
            "fill_draw": live / (32 * wdraw) if wdraw else 0.0,
            "fill_sorted": live / (32 * wsort) if wsort else 0.0}


def im_spread_mc(graph: Graph, seeds, R: int, seed: int = 1):
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    mean, se = ctypes.c_double(), ctypes.c_double()
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    graph.ctx.check(graph.ctx.lib.im_spread_mc(graph.handle, _p(s, ctypes.c_int32), s.shape[0], int(R),
                                               _u64(seed), ctypes.byref(mean), ctypes.byref(se),
                                               ctypes.byref(a), ctypes.byref(b)))
    return {"mean": mean.value, "stderr": se.value, "sum": int(a.value), "sumsq": int(b.value)}


class Batch:
    def __init__(self, ctx: Context, handle, ns):
        self.ctx, self.handle, self.ns = ctx, handle, list(ns)

    def free(self):
        if self.handle:
            self.ctx.lib.im_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def im_batch_load(ctx: Context, graphs, p) -> Batch:
    """graphs: objects with rowptr / col arrays (int32); p: uniform IC probability per graph."""
    G = len(graphs)
    rps = [np.ascontiguousarray(g.rowptr, dtype=np.int32) for g in graphs]
    cols = [np.ascontiguousarray(g.col if len(g.col) else np.zeros(1), dtype=np.int32) for g in graphs]
    n = np.array([r.shape[0] - 1 for r in rps], dtype=np.int32)
    m = np.array([len(g.col) for g in graphs], dtype=np.int64)
    P32 = ctypes.POINTER(ctypes.c_int32)
    rp_arr = (P32 * G)(*[_p(r, ctypes.c_int32) for r in rps])
    col_arr = (P32 * G)(*[_p(c, ctypes.c_int32) for c in cols])
    pf = np.ascontiguousarray(p, dtype=np.float32)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.im_batch_load(ctx.handle, G, _p(n, ctypes.c_int32), _p(m, ctypes.c_int64),
                                    rp_arr, col_arr, _p(pf, ctypes.c_float), ctypes.byref(h)))
    return Batch(ctx, h, n.tolist())


def im_batch_select_seeds(batch: Batch, J, K, seed: int = 2410, rebuild_eps: float = 0.01) -> list:
    """Alg. 4 on every graph of the batch; returns one dict(seeds, score, est) per graph."""
    J = np.ascontiguousarray(J, dtype=np.int32)
    K = np.ascontiguousarray(K, dtype=np.int32)
    tot = int(K.sum())
    seeds = np.empty(tot, dtype=np.int32)
    score = np.empty(tot, dtype=np.float64)
    est = np.empty(tot, dtype=np.float64)
    batch.ctx.check(batch.ctx.lib.im_batch_select_seeds(
        batch.handle, _p(J, ctypes.c_int32), _p(K, ctypes.c_int32), _u64(seed), float(rebuild_eps),
        _p(seeds, ctypes.c_int32), _p(score, ctypes.c_double), _p(est, ctypes.c_double)))
    out, o = [], 0
    for k in K.tolist():
        out.append({"seeds": seeds[o:o + k].copy(), "score": score[o:o + k].copy(), "est": est[o:o + k].copy()})
        o += k
    return out


def im_last_stats(ctx: Context) -> dict:
    s = im_stats()
    ctx.check(ctx.lib.im_last_stats(ctx.handle, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in im_stats._fields_}


def im_ctx_set_timing(ctx: Context, enable: bool = True):
    ctx.check(ctx.lib.im_ctx_set_timing(ctx.handle, 1 if enable else 0))


def im_ctx_set_tuning(ctx: Context, tuning: dict | None = None):
    """Schedule knobs (heavy_indeg, light_batches, grid_blocks, check_every); None = defaults."""
    if tuning is None:
        ctx.check(ctx.lib.im_ctx_set_tuning(ctx.handle, None))
        return
    t = im_tuning()
    cur = im_ctx_get_tuning(ctx)
    cur.update(tuning)
    for k, _ in im_tuning._fields_:
        setattr(t, k, int(cur[k]))
    ctx.check(ctx.lib.im_ctx_set_tuning(ctx.handle, ctypes.byref(t)))


DEFAULT_BARRIER_WAIT_NS = 2_000_000_000
DEFAULT_MAX_LEVELS = 16382


def im_ctx_set_limits(ctx: Context, barrier_wait_ns: int = DEFAULT_BARRIER_WAIT_NS,
                      max_levels: int = DEFAULT_MAX_LEVELS):
    """Bounds of the device-side waits (grid barrier wait, levels per phase)."""
    ctx.check(ctx.lib.im_ctx_set_limits(ctx.handle, _u64(barrier_wait_ns), int(max_levels)))


def im_ctx_get_tuning(ctx: Context) -> dict:
    t = im_tuning()
    ctx.check(ctx.lib.im_ctx_get_tuning(ctx.handle, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in im_tuning._fields_}


def im_ctx_set_trace(ctx: Context, enable: bool = True):
    ctx.check(ctx.lib.im_ctx_set_trace(ctx.handle, 1 if enable else 0))


def im_last_trace(ctx: Context) -> np.ndarray:
    """Per-launch records of the last call: structured array (kind, level, count, edges, ms)."""
    n = int(ctx.lib.im_last_trace(ctx.handle, None, 0))
    buf = (im_trace_rec * max(n, 1))()
    ctx.lib.im_last_trace(ctx.handle, buf, n)
    dt = np.dtype([("kind", np.int32), ("level", np.int32), ("count", np.int64),
                   ("edges", np.int64), ("ms", np.float64)])
    return np.frombuffer(bytes(buf), dtype=dt, count=n).copy()


def im_ctx_bytes_in_use(ctx: Context) -> int:
    return int(ctx.lib.im_ctx_bytes_in_use(ctx.handle))


def im_ctx_bytes_peak(ctx: Context) -> int:
    return int(ctx.lib.im_ctx_bytes_peak(ctx.handle))


class Server:
    """Query server over resident graphs (im_server_*): concurrent selections,
    each on its own worker stream, admitted under a device-memory budget."""

    def __init__(self, device: int = 0, slots: int = 8, hbm_budget_bytes: int = 0, max_bypass: int = 4):
        self.lib = load_library()
        cfg = im_server_config(int(device), int(slots), int(hbm_budget_bytes), int(max_bypass))
        h = ctypes.c_void_p()
        st = self.lib.im_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise IMError(st, "im_server_create")
        self.handle = h
        self.graphs: list = []
        self._live: dict = {}

    def _check(self, st: int, what: str):
        if st != 0:
            raise IMError(st, what)

    def add_graph(self, graph: Graph) -> int:
        gid = ctypes.c_int32()
        self._check(self.lib.im_server_add_graph(self.handle, graph.handle, ctypes.byref(gid)),
                    "im_server_add_graph")
        self.graphs.append(graph)  # the graph must outlive the server
        return gid.value

    def query_bytes(self, graph: int, J: int, K: int) -> int:
        b = ctypes.c_uint64()
        self._check(self.lib.im_server_query_bytes(self.handle, int(graph), int(J), int(K), ctypes.byref(b)),
                    "im_server_query_bytes")
        return int(b.value)

    def submit(self, graph: int, K: int, J: int, model: dict | None = None, seed: int = 2410,
               rebuild_eps: float = 0.01) -> int:
        q = im_query()
        q.graph, q.K, q.J = int(graph), int(K), int(J)
        mdl = _model(model, [])
        if mdl is None:
            q.model.kind = -1
        else:
            q.model = mdl
        q.seed = _u64(seed)
        q.rebuild_eps = float(rebuild_eps)
        seeds = np.empty(K, dtype=np.int32)
        score = np.empty(K, dtype=np.float64)
        est = np.empty(K, dtype=np.float64)
        t = ctypes.c_int64()
        self._check(self.lib.im_server_submit(self.handle, ctypes.byref(q), _p(seeds, ctypes.c_int32),
                                              _p(score, ctypes.c_double), _p(est, ctypes.c_double),
                                              ctypes.byref(t)), "im_server_submit")
        self._live[t.value] = (seeds, score, est)  # the worker writes these until wait returns
        return t.value

    def wait(self, ticket: int, timeout_ms: float = -1.0) -> dict:
        r = im_query_result()
        self._check(self.lib.im_server_wait(self.handle, int(ticket), float(timeout_ms), ctypes.byref(r)),
                    "im_server_wait")
        seeds, score, est = self._live.pop(ticket)
        out = {k: getattr(r, k) for k in ("ticket", "status", "slot", "t_submit_ms", "t_start_ms",
                                          "t_done_ms", "ms_select", "bytes")}
        out["error"] = r.error.decode(errors="replace")
        out.update(seeds=seeds, score=score, est=est)
        return out

    def stats(self) -> dict:
        s = im_server_stats()
        self._check(self.lib.im_server_get_stats(self.handle, ctypes.byref(s)), "im_server_get_stats")
        return {k: getattr(s, k) for k, _ in im_server_stats._fields_}

    def clock_ms(self) -> float:
        return float(self.lib.im_server_clock_ms())

    def close(self):
        if self.handle:
            self.lib.im_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
