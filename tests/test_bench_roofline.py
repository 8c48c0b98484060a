"""The benchmark's roofline numerator is reproducible from the counts it
prints: per frontier vertex 8 + J bytes (row bounds and the register row), per
examined in-edge 4 + t (t = 4 for stored per-edge thresholds, explicit weights
only), per changed vertex J, per live 16-simulation chunk 16; bucket levels per
queued bucket 8 + 16, per list entry 4 + t + 16, per changed bucket 16.  The
DRAM traffic figure is reported only while the propagation kernels' source is
the one it was captured from.  CPU only."""
import hashlib
import json
import os

import bench

STATS = {"sweep_vertices": 1000, "sweep_edges": 20000, "sweep_changed": 300, "sweep_chunks": 50000,
         "sweep_buckets": 7, "sweep_bucket_entries": 11, "sweep_changed_buckets": 5}


def test_alg_bytes_from_units():
    for J in (16, 256, 512, 1024):
        for kind, t in (("wc", 0), ("trivalency", 0), ("uniform", 0), ("explicit", 4)):
            r = bench.alg_bytes_terms(STATS, J, kind)
            assert r["per_unit"] == {"frontier_vertices": 8 + J, "in_edges": 4 + t, "changed_vertices": J,
                                     "live_16sim_chunks": 16, "frontier_buckets": 24,
                                     "bucket_entries": 20 + t, "changed_buckets": 16}
            want = (1000 * (8 + J) + 20000 * (4 + t) + 300 * J + 50000 * 16 + 7 * 24 + 11 * (20 + t) + 5 * 16)
            assert r["bytes"] == want
            assert r["units"]["in_edges"] == 20000 and r["units"]["live_16sim_chunks"] == 50000


def test_traffic_record_follows_the_frontier_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_2410_14047_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "im_frontier.cu").write_bytes(b"kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    rec = {"rmat24": {"traffic_bytes_per_launch": 1.5e9, "frontier_source_sha256": sha}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("rmat24") == 1.5e9
    assert bench.ncu_traffic("rmat20") is None  # no capture for this workload
    (src / "im_frontier.cu").write_bytes(b"kernel v2")  # the kernel changed since the capture
    assert bench.ncu_traffic("rmat24") is None


def test_committed_traffic_record_is_scaled_by_algorithmic_bytes():
    # the full workload's figure is the quarter-size capture scaled by the
    # ratio of the two launches' algorithmic bytes
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = json.load(open(os.path.join(root, "profiles", "ncu_traffic.json")))
    r22, r24 = rec["rmat22"], rec["rmat24"]
    assert r22["frontier_source_sha256"] == r24["frontier_source_sha256"]
    assert abs(r24["traffic_bytes_per_launch"] / r24["alg_bytes_per_launch"] -
               r22["traffic_bytes_per_launch"] / r22["alg_bytes_per_launch"]) < 1e-9
