"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test names what fixes the expected value: a published check vector, a
closed form, a library routine, brute force on a tiny input, or a hand-worked
example from the paper.
"""
import os
import statistics
import struct

import networkx as nx
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import mc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _murmur_vectors():
    out = []
    for line in open(os.path.join(GOLDEN, "murmur3_x86_32_vectors.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, s, e = line.split()
        out.append((b"" if k == "-" else bytes.fromhex(k), int(s, 16), int(e, 16)))
    return out


# --- hash and RNG primitives ------------------------------------------------

@pytest.mark.parametrize("key,seed,expected", _murmur_vectors())
def test_murmur3_published_vectors(key, seed, expected):
    assert O.murmur3_32(key, seed) == expected


def test_splitmix64_published_vector():
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) if l[0].isdigit()]
    expected = np.array([int(x) for x in lines], dtype=np.uint64)
    assert (O.splitmix64(1234567, 5) == expected).all()
    # the input generators carry their own SplitMix64; it must agree too
    assert (W.splitmix_outputs(1234567, 5) == expected).all()


def test_rank_is_leading_zeros_of_published_hashes():
    # Murmur3(LE32(0), 0) = 0x2362F9DE -> 2 leading zeros; Murmur3(21 43 65 87, 0)
    # = 0xF55B516B -> 0; with seed 0x5082EDEE the same key gives 0x2362F9DE -> 2;
    # Murmur3(FF FF FF FF, 0) = 0x76293B50 -> 1 (Eq. sketch-init: clz of h_j(u)).
    assert O.rank(0, 0) == 2
    u = struct.unpack("<i", bytes.fromhex("21436587"))[0]
    assert O.rank(u, 0) == 0
    assert O.rank(u, 0x5082EDEE) == 2
    assert O.rank(-1, 0) == 1


def test_rank_distribution_is_geometric():
    # clz of a uniform 32-bit hash: P(r >= k) = 2^-k
    ranks = np.array([O.rank(u, s) for u in range(4000) for s in (1, 77, 0xDEADBEEF)])
    N = ranks.size
    for k in range(1, 7):
        p = 2.0 ** -k
        got = (ranks >= k).sum()
        assert abs(got - N * p) < 5 * np.sqrt(N * p * (1 - p)), k


def test_edge_hash_key_layout():
    # Eq. (hash): Murmur3(u || v) mod 2^31 with u, v as little-endian int32
    for u, v in [(0, 1), (1, 0), (123456, 7), (2**31 - 1, 5), (5, 2**24)]:
        key = struct.pack("<ii", u, v)
        assert O.edge_hash(u, v) == O.murmur3_32(key, 0) & 0x7FFFFFFF
    assert O.edge_hash(3, 4) != O.edge_hash(4, 3)


def test_draw_sims_sorted_pairs_of_splitmix_stream():
    for seed, J in [(2410, 64), (1, 1024), (99, 16)]:
        X, salt = O.draw_sims(seed, J)
        z = W.splitmix_outputs(seed, J)  # independent implementation
        rawX = (z & np.uint64(0x7FFFFFFF)).astype(np.uint32)
        rawS = (z >> np.uint64(32)).astype(np.uint32)
        order = np.argsort(rawX, kind="stable")
        assert (X == rawX[order]).all() and (salt == rawS[order]).all()
        assert (np.diff(X.astype(np.int64)) >= 0).all() and X.max() < 2**31


# --- thresholds and the live test ------------------------------------------------

def test_threshold_hand_worked_values():
    # fp32(0.01) = 10737418 * 2^-30 -> floor(* 2^31) = 21474836, etc.
    assert O.prob_threshold(0.01) == 21474836
    assert O.prob_threshold(0.005) == 10737418
    assert O.prob_threshold(0.1) == 214748368
    assert O.prob_threshold(0.001) == 2147483
    assert O.prob_threshold(1.0) == 2**31
    assert O.prob_threshold(0.0) == 0
    assert O.prob_threshold(0.5) == 2**30


def test_threshold_models():
    # v=0 has in-degree 1, v=1 in-degree 2, v=2 in-degree 3, v=3 in-degree 4
    g = W.from_edges(8, [(4, 0), (4, 1), (5, 1), (4, 2), (5, 2), (6, 2),
                         (4, 3), (5, 3), (6, 3), (7, 3)])
    thr = O.thresholds(g, {"kind": "wc"})
    by_target = dict(zip(g.col.tolist(), thr.tolist()))
    # fp32(1/3) = 0.3333333432674408 -> 715827904
    assert by_target == {0: 2**31, 1: 2**30, 2: 715827904, 3: 2**29}
    assert (O.thresholds(g, {"kind": "uniform", "p": 0.01}) == 21474836).all()
    w = np.linspace(0, 1, g.m).astype(np.float32)
    assert (O.thresholds(g, {"kind": "explicit", "w": w}) ==
            [O.prob_threshold(x) for x in w]).all()


def test_trivalency_classes_uniform():
    g = W.rmat(12, 8, seed=3)
    thr = O.thresholds(g, {"kind": "trivalency", "seed": 2410})
    vals, cnt = np.unique(thr, return_counts=True)
    assert set(vals.tolist()) == {214748368, 21474836, 2147483}
    exp = g.m / 3
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    assert chi2 < 20  # 2 dof


def test_live_fraction_matches_probability():
    g = W.erdos_renyi(2000, 20000, seed=4)
    X, _ = O.draw_sims(7, 256)
    for p in (0.01, 0.1, 0.37):
        t = O.prob_threshold(p)
        h = np.array([O.edge_hash(u, v) for u in range(g.n)
                      for v in g.col[g.rowptr[u]:g.rowptr[u + 1]]], dtype=np.uint32)
        live = ((X[None, :] ^ h[:, None]) < t).sum()
        N = h.size * X.size
        q = t / 2**31
        # per-edge hashes are shared by the 256 simulations of an edge, so the
        # count is a sum of m independent Binomial(J, q)-like terms; 6 sigma of
        # the binomial bound is generous for that mild dependence
        assert abs(live - N * q) < 6 * np.sqrt(N * q * (1 - q) * 4), p


# --- sketch builds --------------------------------------------------------------

def _small_graphs():
    return [W.erdos_renyi(200, 1200, seed=1), W.rmat(8, 8, seed=2),
            W.from_edges(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 3), (5, 0)])]


@pytest.mark.parametrize("model", [{"kind": "uniform", "p": 0.35}, {"kind": "wc"},
                                   {"kind": "trivalency", "seed": 5}])
def test_three_builds_agree(model):
    rng = np.random.default_rng(0)
    for g in _small_graphs():
        thr = O.thresholds(g, model)
        for J in (16, 64):
            X, salt = O.draw_sims(J * 31 + g.n, J)
            vis = np.where(rng.random((g.n, J)) < 0.2, 0xFF, 0).astype(np.uint8)
            M1 = O.build_bruteforce(g, thr, J, X, salt, vis.copy())
            M2, sweeps = O.build_jacobi(g, thr, J, X, salt, vis.copy())
            M3 = O.build_reverse(g, thr, J, X, salt, vis.copy())
            assert (M1 == M2).all() and (M1 == M3).all()
            assert ((M1 == 0xFF) == (vis == 0xFF)).all()


def _ranks(n, salt):
    return np.array([[O.rank(u, s) for s in salt] for u in range(n)], dtype=np.uint8)


def test_closed_form_w0_registers_are_own_ranks():
    g = W.erdos_renyi(100, 600, seed=9)
    X, salt = O.draw_sims(3, 32)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.0})
    M, sweeps = O.build_jacobi(g, thr, 32, X, salt)
    assert (M == _ranks(g.n, salt)).all() and sweeps == 1


def test_closed_form_w1_path_cycle_star():
    J = 32
    X, salt = O.draw_sims(5, J)
    path = W.from_edges(10, [(i, i + 1) for i in range(9)])
    R = _ranks(10, salt)
    M = O.build_reverse(path, O.thresholds(path, {"kind": "uniform", "p": 1.0}), J, X, salt)
    suffix_max = np.maximum.accumulate(R[::-1], axis=0)[::-1]
    assert (M == suffix_max).all()
    cyc = W.from_edges(7, [(i, (i + 1) % 7) for i in range(7)])
    M = O.build_jacobi(cyc, O.thresholds(cyc, {"kind": "uniform", "p": 1.0}), J, X, salt)[0]
    assert (M == _ranks(7, salt).max(axis=0)[None, :]).all()
    star = W.from_edges(9, [(0, i) for i in range(1, 9)])
    R = _ranks(9, salt)
    M = O.build_bruteforce(star, O.thresholds(star, {"kind": "uniform", "p": 1.0}), J, X, salt)
    assert (M[0] == R.max(axis=0)).all() and (M[1:] == R[1:]).all()
    # a visited middle vertex of the path cuts it (visited registers block reach)
    vis = np.zeros((10, J), np.uint8)
    vis[4, :] = 0xFF
    M = O.build_reverse(path, O.thresholds(path, {"kind": "uniform", "p": 1.0}), J, X, salt, vis)
    R = _ranks(10, salt)
    assert (M[4] == 0xFF).all()
    assert (M[:4] == np.maximum.accumulate(R[:4][::-1], axis=0)[::-1]).all()
    assert (M[5:] == np.maximum.accumulate(R[5:][::-1], axis=0)[::-1]).all()


def test_build_invariants_mid_graph():
    g = W.rmat(12, 8, seed=11)
    model = {"kind": "wc"}
    thr = O.thresholds(g, model)
    J = 64
    X, salt = O.draw_sims(17, J)
    M = O.build_reverse(g, thr, J, X, salt)
    R = _ranks(g.n, salt)
    assert (M >= R).all()
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    h = np.array([O.edge_hash(u, v) for u, v in zip(src, g.col)], dtype=np.uint32)
    live = (X[None, :] ^ h[:, None]) < thr[:, None]
    Mu, Mv = M[src], M[g.col]
    assert (Mu[live] >= Mv[live]).all()  # Alg. 2 fixpoint: M_u >= M_v on live edges


# --- estimate, pick, cover ------------------------------------------------------

def test_estimate_is_harmonic_mean_over_phi():
    rng = np.random.default_rng(1)
    for J in (16, 64, 1024):
        M = rng.integers(0, 33, size=(5, J)).astype(np.uint8)
        M[0, : J // 4] = 0xFF  # visited registers count like rank 0 (2^0)
        S = O.sums(M)
        for u in range(5):
            vals = [2.0 ** (0 if r == 0xFF else int(r)) for r in M[u]]
            h = statistics.harmonic_mean(vals)
            assert O.estimate(J, S[u]) == pytest.approx(h / O.PHI, rel=1e-12)


def test_sums_exact_extremes():
    J = 1024
    assert O.sums(np.zeros((1, J), np.uint8))[0] == J * 2**32
    assert O.sums(np.full((1, J), 0xFF, np.uint8))[0] == J * 2**32
    assert O.sums(np.full((1, J), 32, np.uint8))[0] == J


def test_pick_ties_and_exclusion():
    S = np.array([5, 3, 3, 9, 3], dtype=np.uint64)
    assert O.pick(S, np.zeros(5, np.uint8)) == 1
    assert O.pick(S, np.array([0, 1, 0, 0, 0], np.uint8)) == 2
    assert O.pick(S, np.array([1, 1, 1, 0, 1], np.uint8)) == 3
    assert O.pick(S, np.ones(5, np.uint8)) == -1


def _live_digraph(g, thr, Xj):
    D = nx.DiGraph()
    D.add_nodes_from(range(g.n))
    for u in range(g.n):
        for e in range(g.rowptr[u], g.rowptr[u + 1]):
            v = int(g.col[e])
            if (int(Xj) ^ O.edge_hash(u, v)) < int(thr[e]):
                D.add_edge(u, v)
    return D


def test_cover_equals_reachability_of_seed_set():
    g = W.erdos_renyi(150, 600, seed=21)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.3})
    J = 16
    X, salt = O.draw_sims(8, J)
    M = O.build_reverse(g, thr, J, X, salt)
    seeds, count = [], 0
    for s in (3, 77, 3, 120):
        count += O.cover(g, thr, J, X, M, s)
        seeds.append(s)
        for j in range(J):
            D = _live_digraph(g, thr, X[j])
            reach = set(seeds)
            for t in seeds:
                reach |= nx.descendants(D, t)
            assert set(np.nonzero(M[:, j] == 0xFF)[0].tolist()) == reach
        assert count == O.count_visited(M)


def test_rebuild_rule_hand_worked():
    # Alg. 4: rebuild iff (score - oldscore) / score > e, score = count / J
    assert O.rebuild_due(100, 0, 1, 0.01)          # first seed: oldscore = 0
    assert not O.rebuild_due(100, 99, 1, 0.01)     # 1% growth is not > 1%
    assert O.rebuild_due(100, 98, 1, 0.01)
    assert O.rebuild_due(6400, 6300, 64, 0.01)
    assert not O.rebuild_due(100, 50, 1, -1.0)     # negative e disables rebuilds


def _greedy_brute(g, thr, J, K, seed, eps):
    """Alg. 4 written out with networkx reachability, tiny graphs only."""
    X, salt = O.draw_sims(seed, J)
    R = _ranks(g.n, salt)
    Ds = [_live_digraph(g, thr, X[j]) for j in range(J)]
    visited = [set() for _ in range(J)]

    def build():
        M = np.zeros((g.n, J), np.uint8)
        for j in range(J):
            sub = Ds[j].subgraph([v for v in range(g.n) if v not in visited[j]])
            for u in range(g.n):
                if u in visited[j]:
                    M[u, j] = 0xFF
                else:
                    M[u, j] = max(R[w, j] for w in nx.descendants(sub, u) | {u})
        return M

    M = build()
    seeds, scores, oldcount = [], [], 0
    for k in range(K):
        S = [sum((2**32) if r == 0xFF else 2 ** (32 - int(r)) for r in M[u]) for u in range(g.n)]
        s = min((u for u in range(g.n) if u not in seeds), key=lambda u: (S[u], u))
        seeds.append(s)
        for j in range(J):
            if s not in visited[j]:
                visited[j] |= {s} | nx.descendants(Ds[j], s)
        for j in range(J):
            for u in visited[j]:
                M[u, j] = 0xFF
        count = sum(len(v) for v in visited)
        scores.append(count / J)
        if k + 1 < K and eps >= 0 and (count / J - oldcount / J) / (count / J) > eps:
            M = build()
            oldcount = count
    return seeds, scores, M


@pytest.mark.parametrize("eps", [0.01, 0.0, -1.0])
def test_select_seeds_matches_bruteforce_greedy(eps):
    g = W.erdos_renyi(60, 240, seed=31)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.3})
    J, K = 16, 6
    seeds, scores, M = _greedy_brute(g, thr, J, K, 123, eps)
    for mode in ("jacobi", "reverse", "bruteforce"):
        r = O.select_seeds(g, thr, J, K, 123, eps, mode)
        assert r["seeds"].tolist() == seeds
        assert r["score"].tolist() == scores
        assert (r["M"] == M).all()
    assert all(b >= a for a, b in zip(scores, scores[1:]))  # sigma monotone (Sec. 2.1)


# --- Monte-Carlo spread -----------------------------------------------------------

def _mean_se(sum_, sumsq, R):
    mean = sum_ / R
    return mean, float(np.sqrt(max(sumsq / R - mean**2, 0.0) / R))


def test_mc_single_edge_closed_form():
    # IC (Sec. 2.1): sigma({u}) = 1 + p for a single edge u -> v
    g = W.from_edges(2, [(0, 1)])
    R = 40000
    for p in (0.01, 0.3):
        thr = O.thresholds(g, {"kind": "uniform", "p": p})
        for fn in (O.spread_ic, O.spread_hash):
            mean, se = _mean_se(*fn(g, thr, [0], R, seed=5), R)
            assert abs(mean - (1 + p)) < 4 * se + 1e-12
        m2, se2 = mc.spread(2, [0], [1], [p], [0], 4000, seed=1)
        assert abs(m2 - (1 + p)) < 4 * se2 + 1e-12


def test_mc_parallel_edges_paper_example():
    # Sec. 2.1: two parallel 0.1 edges merge into one edge of 1-(1-0.1)^2 = 0.19
    m_par, se_par = mc.spread(2, [0, 0], [1, 1], [0.1, 0.1], [0], 40000, seed=2)
    assert abs(m_par - 1.19) < 4 * se_par
    g = W.from_edges(2, [(0, 1)])
    thr = O.thresholds(g, {"kind": "explicit", "w": np.array([0.19], np.float32)})
    R = 100000
    mean, se = _mean_se(*O.spread_ic(g, thr, [0], R, seed=9), R)
    assert abs(mean - 1.19) < 4 * se


def test_mc_two_hop_closed_form():
    # path u -> v -> w with independent coins: sigma({u}) = 1 + p + p^2
    g = W.from_edges(3, [(0, 1), (1, 2)])
    p = 0.4
    thr = O.thresholds(g, {"kind": "uniform", "p": p})
    R = 100000
    mean, se = _mean_se(*O.spread_ic(g, thr, [0], R, seed=3), R)
    assert abs(mean - (1 + p + p * p)) < 4 * se


def test_mc_deterministic_reach():
    g = W.rmat(9, 4, seed=6)
    thr = O.thresholds(g, {"kind": "uniform", "p": 1.0})
    D = nx.DiGraph()
    D.add_nodes_from(range(g.n))
    for u in range(g.n):
        for v in g.col[g.rowptr[u]:g.rowptr[u + 1]]:
            D.add_edge(u, int(v))
    seeds = [0, 5, 300]
    reach = set(seeds)
    for s in seeds:
        reach |= nx.descendants(D, s)
    for fn in (O.spread_ic, O.spread_hash):
        s, sq = fn(g, thr, seeds, 50, seed=1)
        assert s == 50 * len(reach) and sq == 50 * len(reach) ** 2


def test_mc_independent_coins_vs_standard_rng():
    g = W.erdos_renyi(300, 1500, seed=12)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.2})
    seeds = [1, 2, 3]
    R = 4000
    m1, se1 = _mean_se(*O.spread_ic(g, thr, seeds, R, seed=3), R)
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m2, se2 = mc.spread(g.n, src, g.col, np.full(g.m, np.float32(0.2)), seeds, R, seed=4)
    assert abs(m1 - m2) < 3.5 * np.sqrt(se1**2 + se2**2)


def test_fused_sampling_correlates_edges():
    # Eq. (hash_prob) reuses one X_r for all edges of simulation r, so two edges
    # whose hashes differ in the top bits are never live together when p < 1/4:
    # the hash-sampled spread is not the IC spread (reason im_spread_mc uses
    # independent coins).  Pick two consecutive edges with differing top-2 bits.
    for a in range(2, 200):
        if (O.edge_hash(0, 1) >> 29) != (O.edge_hash(1, a) >> 29):
            break
    g = W.from_edges(a + 1, [(0, 1), (1, a)])
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.2})
    R = 20000
    s, sq = O.spread_hash(g, thr, [0], R, seed=1)
    # every simulation reaches 1 or 2 vertices (never a): then sum r^2 - 3 sum r + 2R = 0
    assert sq - 3 * s + 2 * R == 0
    # while under independent coins a is reached w.p. p^2 = 0.04
    s_ic, sq_ic = O.spread_ic(g, thr, [0], R, seed=1)
    assert sq_ic - 3 * s_ic + 2 * R > 0


def test_score_equals_hash_sampled_spread():
    # Alg. 4 score = Count(M,-1)/J = mean over the J simulations of |reach(S)|
    g = W.erdos_renyi(400, 2400, seed=13)
    thr = O.thresholds(g, {"kind": "uniform", "p": 0.15})
    J, K = 64, 5
    r = O.select_seeds(g, thr, J, K, 77, 0.01, "reverse")
    for k in range(K):
        s, _ = O.spread_hash(g, thr, r["seeds"][: k + 1], J, seed=77)
        assert s == round(r["score"][k] * J)


# --- single-register and single-simulation checkers -----------------------------
# orc_register_entry and orc_reach_mark check full-size GPU runs one register or
# one simulation at a time; here they are pinned to networkx reachability on the
# live subgraph of each simulation (Eq. hash_prob), not to the oracle's builds.

def _pin_models(g):
    rng = np.random.default_rng(g.n)
    return [{"kind": "uniform", "p": 0.35}, {"kind": "wc"}, {"kind": "trivalency", "seed": 5},
            {"kind": "explicit", "w": rng.uniform(0, 0.6, g.m).astype(np.float32)},
            {"kind": "target", "w": rng.uniform(0, 0.6, g.n).astype(np.float32)}]


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_register_entry_equals_reach_max_of_live_subgraph(gi):
    # Sec. 2.3 / Alg. 2 fixpoint: M[u][j] = max rank over the vertices reachable
    # from u along edges live in simulation j, avoiding visited vertices; a
    # visited u reads 0xFF (Sec. 3.1)
    g = _small_graphs()[gi]
    rng = np.random.default_rng(40 + gi)
    J = 16
    X, salt = O.draw_sims(90 + gi, J)
    R = _ranks(g.n, salt)
    for model in _pin_models(g):
        thr = O.thresholds(g, model)
        vis = np.where(rng.random((g.n, J)) < 0.15, 0xFF, 0).astype(np.uint8)
        for j in range(J):
            D = _live_digraph(g, thr, X[j])
            keep = [v for v in range(g.n) if vis[v, j] == 0]
            sub = D.subgraph(keep)
            for u in range(g.n):
                if vis[u, j]:
                    want = 0xFF
                else:
                    want = max(int(R[w, j]) for w in nx.descendants(sub, u) | {u})
                got = O.register_entry(g, thr, X[j], salt[j], u, vis[:, j])
                assert got == want, (model["kind"], j, u)
            # without visited marks: reach over the whole live subgraph
            for u in range(0, g.n, 7):
                want = max(int(R[w, j]) for w in nx.descendants(D, u) | {u})
                assert O.register_entry(g, thr, X[j], salt[j], u) == want


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_reach_mark_equals_networkx_descendants(gi):
    # Alg. 3 cascade: the vertices reachable from the seed set along edges live
    # in simulation j, the seeds included
    g = _small_graphs()[gi]
    rng = np.random.default_rng(70 + gi)
    J = 16
    X, _ = O.draw_sims(5 + gi, J)
    for model in _pin_models(g):
        thr = O.thresholds(g, model)
        for j in range(J):
            D = _live_digraph(g, thr, X[j])
            k = int(rng.integers(1, 4))
            seeds = rng.integers(0, g.n, size=k).tolist() + [int(rng.integers(0, g.n))] * 2  # repeats
            reach = set(seeds)
            for s in seeds:
                reach |= nx.descendants(D, s)
            mark = O.reach_mark(g, thr, X[j], seeds)
            assert set(np.nonzero(mark)[0].tolist()) == reach, (model["kind"], j)
    assert not O.reach_mark(g, O.thresholds(g, {"kind": "wc"}), X[0], []).any()


def test_thresholds_per_target_hand_worked():
    # per-target model: every edge into v fires with w[v] (Sec. 2.1 with a
    # per-vertex probability); fixed point floor(fp32(w) * 2^31)
    g = W.from_edges(7, [(6, 0), (5, 0), (6, 1), (6, 2), (0, 3), (1, 3), (6, 4), (6, 5), (3, 5)])
    w = np.array([0.01, 0.1, 0.5, 1.0, 0.0, 1.0 / 3.0, 0.9], np.float32)
    thr = O.thresholds(g, {"kind": "target", "w": w})
    by_target = {}
    for e, v in enumerate(g.col.tolist()):
        by_target.setdefault(v, set()).add(int(thr[e]))
    # fp32(0.01) -> 21474836, fp32(0.1) -> 214748368, 0.5 -> 2^30, 1 -> 2^31,
    # 0 -> 0, fp32(1/3) = 0.3333333432674408 -> 715827904
    assert by_target == {0: {21474836}, 1: {214748368}, 2: {2**30}, 3: {2**31}, 4: {0},
                         5: {715827904}}
    # weighted cascade is the per-target case w[v] = fp32(1 / indeg(v))
    h = W.rmat(9, 8, seed=4)
    indeg = np.bincount(h.col, minlength=h.n)
    wv = np.array([1.0 / d if d else 0.0 for d in indeg], np.float32)
    assert (O.thresholds(h, {"kind": "target", "w": wv}) == O.thresholds(h, {"kind": "wc"})).all()
