#!/usr/bin/env python
"""Benchmark of the sketch-based IM hot path (one K-seed selection per step).

A step is one call of im_select_seeds on the large workload: R-MAT scale 24
(16.7M vertices, edge factor 16, a/b/c = 0.57/0.19/0.19, duplicates and
self-loops removed, 263M edges), trivalency IC (p in {0.1, 0.01, 0.001} per
edge by hash), J = 512 simulations (8.6 GB of registers), K = 50 seeds,
rebuild threshold e = 0.01 (the paper's Table 3 setting at Sinaweibo scale;
synthetic because the SNAP graphs are not available).  --workload rmat20 or
er10k selects the mid-size or tiny workload.  Covers every step of the
method: draws, fill, propagation to the fixpoint, estimate + argmax, cover,
count, rebuilds.

Metric: K-seed selections per second (the inverse of time-to-K-seeds),
whole job: with --gpus N every rank runs an independent replica (the path
does not shard on one GPU), value = N * steps / max-over-ranks time.  On one
GPU the line also carries the batched and served forms (nested "forms" key;
--no-forms leaves them out) and the oracle on the host cores (cpu_baseline).

--impl reference times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-K-seeds (K-seed selections/s)"
UNIT = "selections/s"
CPU_SAMPLE_J = 16
ORACLE_CALIBRATION = os.path.join(ROOT, "profiles", "oracle_calibration.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat24")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--mode", default="select", choices=["select", "build", "fillrate", "trace"],
                    help="select: the benchmark; build: time im_sketch_build only (profiling); "
                         "fillrate: warp fill rate of the live tests, draw order vs sorted X (Table 6 analogue); "
                         "trace: per-level records of one selection (frontier sizes, edges, duration)")
    ap.add_argument("--batch-graphs", type=int, default=512,
                    help="graphs of the batched workload (--workload batched)")
    ap.add_argument("--tuning", default="",
                    help="JSON schedule knobs passed to im_ctx_set_tuning (profiling and sweeps)")
    ap.add_argument("--queries", type=int, default=400,
                    help="queries of the served workload (--workload served)")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="mean Poisson arrival rate of the served workload, queries/s")
    ap.add_argument("--slots", type=int, default=8,
                    help="concurrent queries of the server (--workload served)")
    ap.add_argument("--quick", action="store_true",
                    help="profiling runs: no clock sampling, end-to-end pass, CPU baseline or forms")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave the batched and served forms out of the plain benchmark line")
    ap.add_argument("--served-carried-rate", type=float, default=10.0,
                    help="arrival rate of the served run below capacity, queries/s")
    ap.add_argument("--calibrate-oracle", action="store_true",
                    help="time one full oracle selection and the oracle sample on this host "
                         "(the factor that scales the sample to a selection)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (replicas: the slowest rank sets the
    whole job's time); x itself when not distributed."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(steps: int, world: int, tmax: float) -> float:
    """Whole-job throughput of `world` independent replicas that each ran
    `steps` steps, the slowest in tmax seconds."""
    return world * steps / tmax


def alg_bytes_terms(st: dict, J: int, model_kind: str) -> dict:
    """Algorithmic bytes of the propagation launches from their device counts,
    by the per-unit figures of the propagation sweep's byte count: per
    frontier vertex 8 (row bounds) + J (its register row), per examined in-edge
    4 (endpoint) + t (a stored per-edge threshold: explicit weights only; the
    other models' thresholds are per target or recomputed), per changed vertex
    J (its row written), per live chunk 1 byte per simulation of the chunk
    (the neighbour's register bytes: 32 per 32-simulation chunk), counted at
    the 16-simulation granularity the kernels work in: 16 per (edge,
    16-simulation chunk) with a simulation where the edge is live, the source
    changed and its register is not visited (a 32-simulation chunk with one
    such half counts 16, not 32).  Levels on (vertex, 16-simulation chunk)
    buckets count the same at 16-simulation granularity: per queued bucket
    8 + 16, per list entry 4 + t + 16, per changed bucket 16.  Hubs pushed by
    per-simulation hash search are not counted (their edges are searched, not
    read)."""
    t = 4 if model_kind == "explicit" else 0
    per_unit = {"frontier_vertices": 8 + J, "in_edges": 4 + t, "changed_vertices": J, "live_16sim_chunks": 16,
                "frontier_buckets": 8 + 16, "bucket_entries": 4 + t + 16, "changed_buckets": 16}
    units = {"frontier_vertices": st["sweep_vertices"], "in_edges": st["sweep_edges"],
             "changed_vertices": st["sweep_changed"], "live_16sim_chunks": st["sweep_chunks"],
             "frontier_buckets": st["sweep_buckets"], "bucket_entries": st["sweep_bucket_entries"],
             "changed_buckets": st["sweep_changed_buckets"]}
    return {"bytes": sum(units[k] * per_unit[k] for k in units), "units": units, "per_unit": per_unit}


def workload_config(wl, g, world):
    return {"workload": wl.name, "n": g.n, "m": g.m, "J": wl.J, "K": wl.K,
            "model": wl.model["kind"], "rebuild_eps": wl.rebuild_eps, "seed": wl.seed,
            "l2": ("inputs larger than L2 (n*J register bytes > 129 MB), no flush" if g.n * wl.J > 129e6
                   else "register matrix fits in L2 (tiny workload), no flush"),
            "replicas": world, "parallelism": f"replicas x{world}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def ncu_traffic(workload):
    """DRAM bytes (read + write) per propagation-phase launch from the
    committed ncu capture, or None when there is none for this workload or
    the frontier kernels' source changed since it was taken."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json"))).get(workload)
        src = open(os.path.join(ROOT, "paper_2410_14047_gb300", "csrc", "im_frontier.cu"), "rb").read()
        if not d or hashlib.sha256(src).hexdigest() != d["frontier_source_sha256"]:
            return None
        return d["traffic_bytes_per_launch"]
    except Exception:
        return None


def oracle_sample(wl, g, thr) -> float:
    """The bounded oracle sample, in seconds: the oracle's first sketch build
    (Alg. 1 fill + Alg. 2 fixpoint by reverse search, its graph set-up
    included) of CPU_SAMPLE_J of the workload's J simulations."""
    import oracle as O
    X, salt = O.draw_sims(wl.seed, CPU_SAMPLE_J)
    t = time.perf_counter()
    O.build_reverse(g, thr, CPU_SAMPLE_J, X, salt)
    return time.perf_counter() - t


def host_key() -> str:
    import platform
    return f"{platform.machine()}-{os.cpu_count()}cpu"


def oracle_factor(workload: str):
    """Seconds of one full oracle selection per second of the sample, measured
    on this kind of host by --calibrate-oracle; (factor, source)."""
    try:
        cal = json.load(open(ORACLE_CALIBRATION))
        e = cal[workload][host_key()]
        return e["full_s"] / e["sample_s"], (f"one full oracle selection measured {e['full_s']:.1f} s against "
                                              f"{e['sample_s']:.1f} s for the sample on {host_key()} "
                                              f"({e.get('when', '?')})")
    except Exception:
        return None, "no calibration for this host: value not scaled (the sample's own rate)"


def oracle_rate(wl, args_workload, t_sample: float):
    """Selections/s of the oracle from a sample time: the sample scaled by the
    calibrated factor, or (no calibration) the sample's own rate, a bound the
    full selection cannot beat."""
    f, src = oracle_factor(args_workload)
    if f is None:
        return 1.0 / t_sample, None, src
    return 1.0 / (t_sample * f), t_sample * f, src


def cpu_baseline(wl, g, args_workload):
    """The oracle, as it stands, on the bounded sample, scaled to selections/s
    of the whole workload by the calibrated factor."""
    import oracle as O
    thr = O.thresholds(g, wl.model)
    dt = oracle_sample(wl, g, thr)
    value, full_s, src = oracle_rate(wl, args_workload, dt)
    return {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": (f"oracle sketch build (fill + fixpoint, graph set-up included) of {CPU_SAMPLE_J} of the "
                       f"{wl.J} simulations on the same graph and model, measured {dt:.2f} s"),
            "extrapolated": full_s is not None,
            "seconds_per_selection": full_s, "scale_source": src}


def run_calibration(args):
    """One full oracle selection and the sample on this host (minutes to
    hours on the large workload): the factor oracle_factor uses."""
    import oracle as O
    import workloads as W
    wl = W.workload(args.workload)
    g = wl.graph()
    thr = O.thresholds(g, wl.model)
    t_s = oracle_sample(wl, g, thr)
    t = time.perf_counter()
    r = O.select_seeds(g, thr, wl.J, wl.K, wl.seed, wl.rebuild_eps, "reverse")
    t_full = time.perf_counter() - t
    golden = None
    gp = os.path.join(ROOT, "tests", "golden", f"select_{args.workload}.json")
    if os.path.exists(gp):
        golden = json.load(open(gp))["seeds"] == r["seeds"].tolist()
    print(json.dumps({"mode": "calibrate-oracle", "workload": args.workload, "host": host_key(),
                      "threads": O.num_threads(), "sample_s": t_s, "full_s": t_full,
                      "rebuilds": int(r.get("rebuilds", -1)), "seeds_match_golden": golden,
                      "when": time.strftime("%Y-%m-%d")}), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W
    wl = W.workload(args.workload)
    g = wl.graph()
    thr = O.thresholds(g, wl.model)
    for _ in range(args.warmup):
        oracle_sample(wl, g, thr)
    times = [oracle_sample(wl, g, thr) for _ in range(args.steps)]
    per = sum(times) / len(times)
    value, full_s, src = oracle_rate(wl, args.workload, per)
    sample = (f"each step: the oracle's sketch build (fill + fixpoint, graph set-up included) of "
              f"{CPU_SAMPLE_J} of the {wl.J} simulations on the same graph and model")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic", "config": workload_config(wl, g, 1),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": sample, "extrapolated": full_s is not None,
                            "seconds_per_selection": full_s, "scale_source": src},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def batched_form(args):
    """Batched form: many uneven Chung-Lu graphs selected in one batched run
    (rounds fused across graphs, schedule from the autotuner) against the
    plain path (one im_select_seeds per graph, sequentially, on resident
    graphs).  Returns the result dict."""
    import numpy as np
    import torch

    import paper_2410_14047_gb300 as im
    from paper_2410_14047_gb300 import autotune
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    G = args.batch_graphs
    t0 = time.perf_counter()
    graphs, p, J, K = W.batched_workload(G, seed=2410)
    gen_s = time.perf_counter() - t0
    ctx = im.im_ctx_create(local)
    im.im_ctx_set_timing(ctx, True)
    t0 = time.perf_counter()
    B = im.im_batch_load(ctx, graphs, p)
    load_s = time.perf_counter() - t0
    # the schedule knobs that matter for the union (bucketed lists or edge
    # scans, batches per claim), autotuned on the whole batch, untimed
    tune = autotune.tune(ctx, lambda: im.im_batch_select_seeds(B, J, K, seed=2410),
                         space={"buckets": [0, 2], "light_batches": [4, 16]}, repeats=1)
    stream = torch.cuda.current_stream()
    steps = max(args.steps, 1)
    for _ in range(max(args.warmup, 1)):
        res = im.im_batch_select_seeds(B, J, K, seed=2410)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        res = im.im_batch_select_seeds(B, J, K, seed=2410)
    ev1.record(stream)
    ev1.synchronize()
    batched_s = ev0.elapsed_time(ev1) / 1e3 / steps
    bstats = im.im_last_stats(ctx)
    B.free()
    # plain path: one query at a time on resident graphs
    solo = [im.im_graph_load(ctx, g.rowptr, g.col, {"kind": "uniform", "p": pg}) for g, pg in zip(graphs, p)]
    torch.cuda.synchronize()
    finish = []
    identical = True
    t0 = time.perf_counter()
    for i, Gs in enumerate(solo):
        r = im.im_select_seeds(Gs, K[i], J[i], seed=2410)
        finish.append(time.perf_counter() - t0)
        identical &= r["seeds"].tolist() == res[i]["seeds"].tolist()
    plain_s = time.perf_counter() - t0
    for Gs in solo:
        Gs.free()
    lat = np.array(finish)
    return {"metric": "batched K-seed selections/s", "value": G / batched_s, "unit": "selections/s",
            "impl": "gb300-batched", "n_gpus": 1, "steps": steps, "ms_per_step": batched_s * 1e3,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic (seeded Chung-Lu graphs)",
            "config": {"workload": f"batched: {G} Chung-Lu graphs gamma 2.1, n U[1k,200k], avg deg U[8,32], "
                                   f"K U[5,50], J {{64,128}}, p U[0.005,0.05]",
                       "graphs": G, "sum_n": int(sum(g.n for g in graphs)), "sum_m": int(sum(g.m for g in graphs)),
                       "sum_K": int(sum(K))},
            "plain": {"value": G / plain_s, "unit": "selections/s", "total_s": plain_s,
                      "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))},
            "batched_latency": {"p50_s": batched_s, "p99_s": batched_s,
                                "note": "every graph of a batch completes with the batch, so p50 = p99 = "
                                        "the batch time; the plain path's latencies count from the start "
                                        "of the sequence"},
            "speedup_vs_plain": plain_s / batched_s,
            "identical_to_plain": bool(identical),
            "autotune": {"tuning": tune["tuning"], "trials": len(tune["trials"])},
            "batched_kernel_ms": {k: bstats[k] for k in ("ms_propagate", "ms_cover_kernels", "ms_pick_kernels",
                                                          "ms_fill_kernels")},
            "generation_s": gen_s, "batch_load_s": load_s}


def run_batched(args):
    out = batched_form(args)
    out["warmup"] = args.warmup
    print(json.dumps(out), flush=True)
    return 0


class ServedSetup:
    """16 resident R-MAT graphs (scales 14-22) loaded once for served runs."""

    def __init__(self, local: int):
        import torch

        import paper_2410_14047_gb300 as im
        import workloads as W
        self.local = local
        t0 = time.perf_counter()
        self.graphs = W.served_graphs(seed=2410)
        self.gen_s = time.perf_counter() - t0
        self.ctx = im.im_ctx_create(local)
        self.loaded = [im.im_graph_load(self.ctx, g.rowptr, g.col, {"kind": "wc"}) for g in self.graphs]
        torch.cuda.synchronize()
        self.warm = False


def served_run(st: ServedSetup, queries: int, rate: float, slots: int, warmup: int, quick: bool):
    """Poisson arrivals of queries against the resident graphs, run by the
    query server (concurrent slots, HBM-budget admission) and, on the same
    arrival sequence, by the plain path one query at a time.  Latency =
    completion - arrival; queries/s = queries / (last completion - first
    arrival).  Returns the result dict."""
    import numpy as np
    import torch

    import paper_2410_14047_gb300 as im
    import workloads as W

    graphs, loaded, local = st.graphs, st.loaded, st.local
    qs = W.served_queries(queries, rate=rate, n_graphs=len(graphs), seed=2410)
    budget = 150 * 10**9
    srv = im.Server(local, slots=slots, hbm_budget_bytes=budget, max_bypass=2 * slots)
    for G in loaded:
        srv.add_graph(G)

    def args_of(q):
        return {k: q[k] for k in ("graph", "K", "J", "model", "seed", "rebuild_eps")}

    if not st.warm:
        warm = W.served_queries(max(warmup, 1) * 4, rate=1e6, n_graphs=len(graphs), seed=99)
        for q in warm:  # module load, pool growth, first launches of each path
            srv.wait(srv.submit(**args_of(q)))
            im.im_select_seeds(loaded[q["graph"]], q["K"], q["J"], model=q["model"], seed=q["seed"])
        torch.cuda.synchronize()
        st.warm = True

    clocks = None if quick else ClockSampler(local)
    if clocks:
        clocks.start()
    # served: submit at the arrival times, collect completions
    t_base = srv.clock_ms() + 50.0
    tickets = []
    for q in qs:
        due = t_base + q["arrival_s"] * 1e3
        while True:
            now = srv.clock_ms()
            if now >= due:
                break
            time.sleep(min(0.002, (due - now) / 1e3))
        tickets.append(srv.submit(**args_of(q)))
    served = [srv.wait(t) for t in tickets]
    sstats = srv.stats()
    s_done = np.array([r["t_done_ms"] for r in served])
    s_start = np.array([r["t_start_ms"] for r in served])
    s_arr = np.array([t_base + q["arrival_s"] * 1e3 for q in qs])
    s_lat = (s_done - s_arr) / 1e3
    s_wait = (s_start - s_arr) / 1e3
    served_s = (s_done.max() - s_arr.min()) / 1e3
    srv.close()
    # plain: one query at a time in arrival order on the same resident graphs
    t_base = srv.clock_ms() + 50.0
    p_done, p_start = [], []
    plain_res = []
    for q in qs:
        due = t_base + q["arrival_s"] * 1e3
        while srv.clock_ms() < due:
            time.sleep(0.001)
        p_start.append(max(due, srv.clock_ms()))
        plain_res.append(im.im_select_seeds(loaded[q["graph"]], q["K"], q["J"], model=q["model"],
                                            seed=q["seed"], rebuild_eps=q["rebuild_eps"]))
        p_done.append(srv.clock_ms())
    p_done = np.array(p_done)
    p_service = p_done - np.array(p_start)
    p_arr = np.array([t_base + q["arrival_s"] * 1e3 for q in qs])
    p_lat = (p_done - p_arr) / 1e3
    p_wait = (np.array(p_start) - p_arr) / 1e3
    plain_s = (p_done.max() - p_arr.min()) / 1e3
    clk = clocks.stop() if clocks else None
    identical = all(r["status"] == 0 and r["seeds"].tolist() == pr["seeds"].tolist()
                    and np.array_equal(r["score"], pr["score"]) for r, pr in zip(served, plain_res))
    N = len(qs)
    out = {"metric": "served IM queries/s (p50/p99 latency, arrival to result)", "value": N / served_s,
           "unit": "queries/s", "impl": "gb300-served", "n_gpus": 1, "higher_is_better": True,
           "dtype": "u8", "data": "synthetic (seeded R-MAT graphs, Poisson arrivals)",
           "config": {"workload": f"served: 16 resident R-MAT graphs scales 14-22 ef 16, {N} queries, "
                                  f"Poisson {rate:g}/s, K {{10,25,50}}, J {{64,256,1024}}, "
                                  "model p=0.01 or WC, 150 GB budget",
                      "queries": N, "rate": rate, "slots": slots, "budget_bytes": budget,
                      "sum_n": int(sum(g.n for g in graphs)), "sum_m": int(sum(g.m for g in graphs))},
           "served": {"value": N / served_s, "total_s": served_s,
                      "p50_s": float(np.percentile(s_lat, 50)), "p99_s": float(np.percentile(s_lat, 99)),
                      "queue_wait_p50_s": float(np.percentile(s_wait, 50)),
                      "running_peak": sstats["running_peak"], "reserved_peak_bytes": sstats["reserved_peak"],
                      "graph_bytes": sstats["graph_bytes"], "bypassed": sstats["bypassed"]},
           "plain": {"value": N / plain_s, "unit": "queries/s", "total_s": plain_s,
                     "p50_s": float(np.percentile(p_lat, 50)), "p99_s": float(np.percentile(p_lat, 99)),
                     "queue_wait_p50_s": float(np.percentile(p_wait, 50)),
                     "service_p50_ms": float(np.percentile(p_service, 50))},
           "speedup_vs_plain": plain_s / served_s,
           "p99_vs_plain": float(np.percentile(p_lat, 99)) / float(np.percentile(s_lat, 99)),
           "identical_to_plain": bool(identical),
           "generation_s": st.gen_s}
    if clk:
        out["clocks"] = clk
    return out


def run_served(args):
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    st = ServedSetup(local)
    print(json.dumps(served_run(st, args.queries, args.rate, args.slots, args.warmup, args.quick)), flush=True)
    return 0


def forms(args):
    """The batched and served forms for the plain benchmark line: the batch
    against plain selections, and the server at an arrival rate both paths can
    carry (latency = service time and overlap) and at the overload rate of the
    served configuration (latency = queueing)."""
    import torch
    out = {"batched": batched_form(args)}
    torch.cuda.empty_cache()
    st = ServedSetup(dist_env()[2])
    out["served_carried"] = served_run(st, max(args.queries // 2, 50), args.served_carried_rate, args.slots,
                                       args.warmup, True)
    out["served_overload"] = served_run(st, args.queries, args.rate, args.slots, args.warmup, True)
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2410_14047_gb300 as im
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = W.workload(args.workload)
    g = wl.graph()
    ctx = im.im_ctx_create(local)
    if args.tuning:
        im.im_ctx_set_tuning(ctx, json.loads(args.tuning))
    G = im.im_graph_load(ctx, g.rowptr, g.col, wl.model)
    im.im_ctx_set_timing(ctx, True)

    if args.mode == "fillrate":
        # the paper's Table 6 setting: J = 1024, uniform w = 0.01 and 0.1; plus weighted cascade
        rows = []
        for model in ({"kind": "uniform", "p": 0.01}, {"kind": "uniform", "p": 0.1}, {"kind": "wc"}):
            r = im.im_fill_rate(G, 1024, seed=wl.seed, model=model)
            rows.append({"model": model, "J": 1024, **r})
        if rank == 0:
            print(json.dumps({"mode": "fillrate", "workload": wl.name, "rows": rows}), flush=True)
        return 0

    if args.mode == "build":
        # profiling mode: sketch builds only (fill + propagation to the fixpoint)
        for _ in range(args.warmup):
            im.im_sketch_build(G, wl.J, wl.seed).free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            im.im_sketch_build(G, wl.J, wl.seed).free()
        torch.cuda.synchronize()
        if rank == 0:
            st = im.im_last_stats(ctx)
            terms = alg_bytes_terms(st, wl.J, wl.model["kind"])
            print(json.dumps({"mode": "build", "workload": wl.name, "steps": args.steps,
                              "ms_per_build": (time.perf_counter() - t0) / max(args.steps, 1) * 1e3,
                              "sweeps": st["sweeps"], "ms_propagate": st["ms_propagate"],
                              "alg_bytes_last_build": terms["bytes"], "units_last_build": terms["units"]}),
                  flush=True)
        return 0

    def step():
        return im.im_select_seeds(G, wl.K, wl.J, seed=wl.seed, rebuild_eps=wl.rebuild_eps)

    if args.mode == "trace":
        # one warm selection, then one traced: every level of every phase
        step()
        im.im_ctx_set_trace(ctx, True)
        r = step()
        tr = im.im_last_trace(ctx)
        st = im.im_last_stats(ctx)
        im.im_ctx_set_trace(ctx, False)
        phases, cur = [], None
        for rec in tr:
            kind = ["propagate", "cover", "affect"][int(rec["kind"])]
            if rec["level"] == 0 or cur is None or kind != cur["kind"]:
                cur = {"kind": kind, "levels": []}
                phases.append(cur)
            cur["levels"].append([int(rec["count"]), int(rec["edges"]), round(float(rec["ms"]), 4)])
        summary = {}
        for ph in phases:
            d = summary.setdefault(ph["kind"], {"phases": 0, "levels": 0, "ms": 0.0})
            d["phases"] += 1
            d["levels"] += len(ph["levels"])
            d["ms"] += sum(x[2] for x in ph["levels"])
        if rank == 0:
            print(json.dumps({"mode": "trace", "workload": wl.name, "seeds": r["seeds"].tolist()[:8],
                              "summary": summary,
                              "propagation_phases": [p["levels"] for p in phases if p["kind"] == "propagate"],
                              "largest_covers": sorted(([round(sum(x[2] for x in p["levels"]), 4), p["levels"]]
                                                        for p in phases if p["kind"] == "cover"),
                                                       key=lambda x: -x[0])[:3],
                              "stats": {k: st[k] for k in ("ms_propagate", "ms_cover_kernels", "ms_pick_kernels",
                                                           "ms_fill_kernels", "builds", "sweeps",
                                                           "cover_levels")}}), flush=True)
        return 0

    # the schedule knobs for this workload: the project's autotuner, untimed
    tuned = None
    if not args.tuning and not args.quick:
        from paper_2410_14047_gb300 import autotune
        tuned = autotune.tune(ctx, step, repeats=1)

    ref_seeds = None
    for _ in range(args.warmup):
        ref_seeds = step()["seeds"].tolist()
    if ref_seeds is None:
        ref_seeds = step()["seeds"].tolist()

    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local) if not args.quick else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    agg = {"alg_bytes_sweep": 0, "ms_propagate": 0.0, "sweep_launches": 0, "launches": 0,
           "builds": 0, "sweeps": 0, "ms_pick_kernels": 0.0, "ms_cover_kernels": 0.0,
           "ms_fill_kernels": 0.0, "cover_levels": 0, "sweep_edges": 0, "sweep_bucket_entries": 0,
           "sweep_vertices": 0, "sweep_changed": 0, "sweep_chunks": 0, "sweep_buckets": 0,
           "sweep_changed_buckets": 0, "sweep_heavy": 0, "sweep_heavy_sims": 0}
    deterministic = True
    ev0.record(stream)
    for _ in range(args.steps):
        r = step()
        st = im.im_last_stats(ctx)
        for k in agg:
            agg[k] += st[k]
        deterministic &= (r["seeds"].tolist() == ref_seeds)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    elapsed = ev0.elapsed_time(ev1) / 1e3
    tmax = max_over_ranks(elapsed, dist, "cuda")

    # end-to-end through the public API with host buffers: pinned host CSR,
    # graph load (H2D copy) + selection + result read-back every step
    rp_pin = torch.from_numpy(g.rowptr).pin_memory()
    col_pin = torch.from_numpy(g.col).pin_memory()
    rp_np, col_np = rp_pin.numpy(), col_pin.numpy()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(0 if args.quick else args.e2e_steps):
        G2 = im.im_graph_load(ctx, rp_np, col_np, wl.model)
        r2 = im.im_select_seeds(G2, wl.K, wl.J, seed=wl.seed, rebuild_eps=wl.rebuild_eps)
        G2.free()
        deterministic &= (r2["seeds"].tolist() == ref_seeds)
    torch.cuda.synchronize()
    e_el = time.perf_counter() - e0
    e_max = max_over_ranks(e_el, dist, "cuda")

    if rank == 0:
        golden = None
        gp = os.path.join(ROOT, "tests", "golden", f"select_{args.workload}.json")
        if os.path.exists(gp):
            golden = json.load(open(gp))["seeds"] == ref_seeds
        peaks = measured_peaks()
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        launches = max(agg["sweep_launches"], 1)
        terms = alg_bytes_terms(agg, wl.J, wl.model["kind"])
        achieved = (terms["bytes"] / 1e9) / (agg["ms_propagate"] / 1e3) if agg["ms_propagate"] else 0.0
        tr = ncu_traffic(args.workload)
        out = {
            "metric": METRIC, "value": replicas_value(args.steps, world, tmax), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded R-MAT standing in for the paper's SNAP graphs)",
            "config": workload_config(wl, g, world),
            "time_to_k_seeds_s": tmax / args.steps,
            # (edge, simulation) pairs the propagation covered: every simulation
            # of an examined in-edge on vertex levels, the 16 of a chunk per list
            # entry on bucket levels
            "register_gteps": (agg["sweep_edges"] * wl.J + agg["sweep_bucket_entries"] * 16)
            / (agg["ms_propagate"] / 1e3) / 1e9 if agg["ms_propagate"] else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": tr,
                         "kernel": "k_phase<%s,kPush> (persistent propagation phase, one launch per build)"
                                   % {"wc": "kWC", "uniform": "kUniform", "trivalency": "kTrivalency",
                                      "explicit": "kExplicit"}[wl.model["kind"]],
                         "alg_bytes_per_launch": terms["bytes"] / launches,
                         "avg_launch_ms": agg["ms_propagate"] / launches,
                         "launches_per_step": agg["sweep_launches"] / args.steps,
                         # the counts behind alg_bytes_per_launch (per launch)
                         "units_per_launch": {k: v / launches for k, v in terms["units"].items()},
                         "bytes_per_unit": terms["per_unit"],
                         "alg_bytes_model_per_launch": agg["alg_bytes_sweep"] / launches,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback"},
            "phase_ms_per_step": {k: agg[k] / args.steps for k in
                                  ("ms_propagate", "ms_pick_kernels", "ms_cover_kernels", "ms_fill_kernels")},
            "counts_per_step": {k: agg[k] / args.steps for k in
                                ("builds", "sweeps", "sweep_launches", "cover_levels", "launches")},
            "gpu_launches": int(agg["launches"]),
            "e2e": {"value": replicas_value(args.e2e_steps, world, e_max) if not args.quick else None, "unit": UNIT,
                    "h2d_bytes_per_step": int(g.rowptr.nbytes + g.col.nbytes),
                    "d2h_bytes_per_step": int(wl.K * (4 + 8 + 8))},
            "clocks": clocks,
            "deterministic": bool(deterministic),
            "seeds_match_oracle_golden": golden,
            "tuning": {"knobs": im.im_ctx_get_tuning(ctx),
                       "source": "autotuner (untimed, before warm-up)" if tuned else
                       ("--tuning" if args.tuning else "defaults")},
        }
        if world == 1 and not args.no_cpu_baseline and not args.quick:
            out["cpu_baseline"] = cpu_baseline(wl, g, args.workload)
        if world == 1 and not args.no_forms and not args.quick:
            del G, ctx
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            out["forms"] = forms(args)
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.calibrate_oracle:
        return run_calibration(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
