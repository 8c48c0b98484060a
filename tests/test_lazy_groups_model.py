"""Host model of the lazy pick over group records: every pick must equal the
plain argmin of (S_u, u) over the unpicked rows (the lowest id on ties).

The model follows the kernels' steps: stored sums lb[u] <= S[u] (the sums only
grow during a selection); per group of G rows a record of the two least stored
pairs of its unpicked rows; a pick takes the runner-up c of the previous pick,
computes S_c fresh, refreshes every unpicked row of each group whose least
recorded pair is below (S_c, c) and records that group again, then takes the
two least pairs over all records; the picked row's group is recorded again
without it.  Random instances with many ties and growing sums; CPU only."""
import numpy as np
import pytest

BIG = np.iinfo(np.int64).max


def group_record(lb, picked, g, G):
    rows = [v for v in range(g * G, min((g + 1) * G, len(lb))) if not picked[v]]
    pairs = sorted((int(lb[v]), v) for v in rows)[:2]
    while len(pairs) < 2:
        pairs.append((BIG, 1 << 30))
    return pairs


def top2(pairs):
    return sorted(pairs)[:2]


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("G", [1, 4, 16])
def test_group_lazy_pick_equals_full_argmin(seed, G):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 120))
    S = rng.integers(0, 12, size=n).astype(np.int64)  # small values: many ties
    picked = np.zeros(n, bool)
    # the first pick reads every row (full pick) and stores every sum
    lb = S.copy()
    ngroups = (n + G - 1) // G
    recs = [group_record(lb, picked, g, G) for g in range(ngroups)]
    full = top2([(int(S[v]), v) for v in range(n)])
    s, cand = full[0][1], full[1][1]
    picked[s] = True
    recs[s // G] = group_record(lb, picked, s // G, G)
    for _ in range(min(n - 1, 40)):
        # a cover and sometimes a rebuild: every sum grows by some amount
        S += rng.integers(0, 4, size=n) * rng.integers(0, 2, size=n)
        assert (lb <= S).all()
        want = min((int(S[v]), v) for v in range(n) if not picked[v])
        # lazy pick over the records
        Sc, uc = (int(S[cand]), cand) if cand < n and not picked[cand] else (0, -1)
        pairs = []
        for g in range(ngroups):
            r = recs[g]
            if r[0] < (Sc, uc):
                for v in range(g * G, min((g + 1) * G, n)):
                    if not picked[v] and (int(lb[v]), v) < (Sc, uc):
                        lb[v] = S[v]
                recs[g] = group_record(lb, picked, g, G)
            pairs += recs[g]
        best = top2(pairs)
        assert best[0] == want, (best, want)
        s, cand = best[0][1], best[1][1]
        picked[s] = True
        recs[s // G] = group_record(lb, picked, s // G, G)
        if picked.all():
            break
