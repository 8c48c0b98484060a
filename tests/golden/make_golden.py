"""Writes the oracle's expected outputs for the named plain-method workloads.

Calls only the oracle (and the seeded input generators for its inputs).
Usage: python tests/golden/make_golden.py er10k rmat20
Output: tests/golden/select_<name>.json (seeds, scores, estimates, rebuilds,
plus SHA-256 digests of the final registers and of the graph).
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.rowptr).tobytes())
    h.update(np.ascontiguousarray(g.col).tobytes())
    return h.hexdigest()


def main(names):
    for name in names:
        wl = W.workload(name)
        g = wl.graph()
        thr = O.thresholds(g, wl.model)
        t = time.time()
        r = O.select_seeds(g, thr, wl.J, wl.K, wl.seed, wl.rebuild_eps, "reverse")
        dt = time.time() - t
        out = {
            "workload": wl.name,
            "n": g.n, "m": g.m, "J": wl.J, "K": wl.K, "seed": wl.seed,
            "rebuild_eps": wl.rebuild_eps, "model": {k: v for k, v in wl.model.items() if k != "w"},
            "graph_sha256": graph_digest(g),
            "seeds": r["seeds"].tolist(),
            "score": [float(x) for x in r["score"]],
            "est": [float(x).hex() for x in r["est"]],
            "rebuilds": r["rebuilds"],
            "registers_sha256": hashlib.sha256(r["M"].tobytes()).hexdigest(),
            "visited": int((r["M"] == 0xFF).sum()),
            "oracle_seconds": round(dt, 1),
            "oracle_threads": O.num_threads(),
        }
        with open(os.path.join(HERE, f"select_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "done in", round(dt, 1), "s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["er10k", "rmat20"])
