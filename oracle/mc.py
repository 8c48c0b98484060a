"""Independent Monte-Carlo spread oracle with a standard RNG (Sec. 5.1).

The paper checks seed-set quality with a separate, unoptimized oracle that
uses standard random number generators and many samples.  This is that
oracle: R independent-cascade simulations from a seed set, each edge
(u, v) firing with probability w(u, v) the first time u is active, coins
drawn from numpy's PCG64.  It supports multigraphs (parallel edges are
independent coins), which lets the tests check the paper's merged-edge
example (Sec. 2.1) directly.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def spread(n: int, src, dst, w, seeds, R: int, seed: int = 0):
    """Mean and standard error of |reach(S)| over R IC simulations.

    src, dst, w: edge list (parallel edges allowed), w float probabilities.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    order = np.argsort(src, kind="stable")
    src, dst, w = src[order], dst[order], w[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, src + 1, 1)
    rowptr = np.cumsum(rowptr)
    rng = np.random.default_rng(seed)
    sizes = np.empty(R, dtype=np.float64)
    seeds = np.unique(np.asarray(seeds, dtype=np.int64))
    for r in range(R):
        active = np.zeros(n, dtype=bool)
        active[seeds] = True
        frontier = seeds
        while frontier.size:
            starts, ends = rowptr[frontier], rowptr[frontier + 1]
            lens = ends - starts
            if lens.sum() == 0:
                break
            idx = np.repeat(starts - np.cumsum(lens) + lens, lens) + np.arange(lens.sum())
            fired = rng.random(idx.size) < w[idx]
            cand = np.unique(dst[idx[fired]])
            cand = cand[~active[cand]]
            active[cand] = True
            frontier = cand
        sizes[r] = active.sum()
    mean = float(sizes.mean())
    se = float(sizes.std(ddof=1) / np.sqrt(R)) if R > 1 else float("inf")
    return mean, se
