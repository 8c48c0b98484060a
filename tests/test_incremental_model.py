"""The incremental rebuild's reasoning, checked on the CPU against the oracle's
full rebuild (Alg. 4 rebuilds every unvisited register: fill, Alg. 1, then
Alg. 2 to the fixpoint).  After covers, a register M[u][j] can change only if
u reaches, in simulation j and through unvisited vertices, a register visited
since the last build; resetting exactly those registers to their own ranks,
taking for each the maximum over its live out-edges, and propagating to the
fixpoint gives the full rebuild's registers.  This is a plain model of the
method the GPU path implements, built from the oracle's primitives."""
import numpy as np

import oracle as O
import workloads as W

VIS = 0xFF


def live_masks(g, thr, X):
    """live[e, j] for every out-edge e = (u -> v): Eq. hash_prob."""
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    h = np.array([O.edge_hash(int(u), int(v)) for u, v in zip(src, g.col)], dtype=np.uint64)
    return src, (X[None, :].astype(np.uint64) ^ h[:, None]) < thr[:, None].astype(np.uint64)


def incremental(M, newly, src, dst, live, salt):
    n, J = M.shape
    # 1. affected: unvisited registers reaching a newly visited one (backwards
    #    over live edges, through unvisited vertices)
    aff = np.zeros_like(newly)
    into = [[] for _ in range(n)]
    for e in range(len(src)):
        into[dst[e]].append(e)
    for j in range(J):
        stack = list(np.nonzero(newly[:, j])[0])
        while stack:
            v = stack.pop()
            for e in into[v]:
                u = src[e]
                if live[e, j] and M[u, j] != VIS and not aff[u, j]:
                    aff[u, j] = True
                    stack.append(u)
    # 2. reset to the own ranks (Alg. 1)
    for u, j in zip(*np.nonzero(aff)):
        M[u, j] = O.rank(int(u), int(salt[j]))
    # 3. pull over the live out-edges
    for e in range(len(src)):
        u, v = src[e], dst[e]
        ok = aff[u] & live[e] & (M[v] != VIS)
        M[u] = np.where(ok, np.maximum(M[u], M[v]), M[u])
    # 4. propagate to the fixpoint from the affected registers only (a push:
    #    a changed register raises its live in-neighbours, which then change)
    changed = aff.copy()
    while changed.any():
        nxt = np.zeros_like(changed)
        for e in range(len(src)):
            u, v = src[e], dst[e]
            ok = changed[v] & live[e] & (M[u] != VIS) & (M[v] != VIS) & (M[v] > M[u])
            if ok.any():
                M[u] = np.where(ok, M[v], M[u])
                nxt[u] |= ok
        changed = nxt
    return M, aff


def test_incremental_rebuild_model_equals_full_rebuild():
    g = W.erdos_renyi(250, 1500, seed=77)
    thr = O.thresholds(g, {"kind": "wc"})
    J = 32
    X, salt = O.draw_sims(5, J)
    src, live = live_masks(g, thr, X)
    dst = g.col.astype(np.int64)
    M = O.build_reverse(g, thr, J, X, salt)
    is_seed = np.zeros(g.n, np.uint8)
    last_build = M == VIS
    affected_seen = 0
    for rnd in range(4):
        # one or two covers between rebuilds (newly visited registers accumulate)
        for _ in range(1 + rnd % 2):
            s = O.pick(O.sums(M), is_seed)
            is_seed[s] = 1
            O.cover(g, thr, J, X, M, s)
        newly = (M == VIS) & ~last_build
        full = O.build_reverse(g, thr, J, X, salt, M.copy())
        inc, aff = incremental(M.copy(), newly, src, dst, live, salt)
        assert np.array_equal(inc, full), rnd
        assert not np.any(aff & (M == VIS))  # visited registers are never reset
        affected_seen += int(aff.sum())
        M = full
        last_build = M == VIS
    assert affected_seen > 0


def test_unaffected_registers_keep_their_values_across_a_rebuild():
    # the registers the search leaves alone are already the full rebuild's
    g = W.erdos_renyi(200, 1100, seed=91)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.2})
    J = 16
    X, salt = O.draw_sims(8, J)
    src, live = live_masks(g, thr, X)
    dst = g.col.astype(np.int64)
    M = O.build_reverse(g, thr, J, X, salt)
    before = M.copy()
    s = O.pick(O.sums(M), np.zeros(g.n, np.uint8))
    O.cover(g, thr, J, X, M, s)
    newly = (M == VIS) & (before != VIS)
    full = O.build_reverse(g, thr, J, X, salt, M.copy())
    _, aff = incremental(M.copy(), newly, src, dst, live, salt)
    keep = ~aff & (M != VIS)
    assert np.array_equal(full[keep], M[keep])
