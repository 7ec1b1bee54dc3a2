"""Benchmark: frontier BFS / SSSP GTEPS on R-MAT scale 24 (edge factor 32,
a/b/c/d = .57/.19/.19/.05, weights U[1,255], seed 1) from 64 sources drawn
uniformly among vertices with out-edges, on one GB300 per rank.

One step = one BFS and one SSSP from each of the rank's 64 sources with the
library's best strategy (workload decomposition).  value = traversed edges
(m_reached per query, summed over every query of every rank) / the max over
ranks of the device time of the K timed steps.  The graph (4.4 GB) is
resident in HBM before timing; it is larger than L2, so no flush is needed.

Also reported: per-strategy timings (BS, EP, WD, NS, HP) on a subset of the
sources, the roofline of the dominant kernel, an end-to-end number through
the host-buffer C-ABI calls, and the CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU runs are query replicas (torchrun, one rank per GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFS/SSSP GTEPS on 1 GB300, % of HBM roofline; batched queries/s, p99 latency"
WORKLOAD = dict(workload="rmat24_ef32_64src", graph="R-MAT scale 24, edge factor 32, a/b/c/d=.57/.19/.19/.05, "
                "self-loops and duplicates removed, weights U[1,255], seed 1", sources=64,
                source_rule="uniform among out-degree>0 vertices, seed 1", kinds=["bfs", "sssp"],
                l2="inputs larger than L2 (CSR 4.4 GB)")
# Compulsory bytes per reached edge / vertex (BFS: col 4 + dst status 4;
# offsets 16 + queue pop 4 + push 4 + level write 4.  SSSP adds the weight
# and the source distance read.)
BYTES = {"bfs": (8, 28), "sssp": (12, 32)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--edge-factor", type=int, default=32)
    ap.add_argument("--sources", type=int, default=64)
    ap.add_argument("--strategy", default="WD")
    ap.add_argument("--compare-sources", type=int, default=4)
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="0: device-resident loop (CUDA graph WHILE); 1: host loop (for per-kernel profiling)")
    ap.add_argument("--kinds", default="bfs,sssp")
    ap.add_argument("--wd-tile", type=int, default=0, help="largest WD tile in list edges (0 = library default)")
    ap.add_argument("--hp-mode", type=int, default=0, help="HP form: 0 sub-iterations, 1 degree-binned")
    ap.add_argument("--ns-mode", type=int, default=0, help="NS form: 0 thread per granule, 1 binned granules")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library default options)")
    ap.add_argument("--no-serve", action="store_true", help="skip the batched-serving measurement")
    ap.add_argument("--serve-queries", type=int, default=1024)
    ap.add_argument("--serve-only", action="store_true", help="run only the batched-serving measurement")
    ap.add_argument("--serve-timeout", type=float, default=120.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def rank_sources(g, per_rank: int, rank: int, world: int):
    """Rank r's sources: its slice of one seeded draw of per_rank x world
    sources (uniform among out-degree > 0 vertices), so the ranks' query
    sets are disjoint and together are the draw a single rank would make
    for the whole job."""
    import graphgen as gg
    all_src = gg.pick_sources(g, per_rank * world, seed=1)
    return all_src[rank * per_rank:(rank + 1) * per_rank]


def combine_ranks(t_ms: float, edges_rank: float, world: int, device: str):
    """Whole-job numbers over the ranks of a replica run: the slowest
    rank's time, the edges every rank traversed, and GTEPS = total edges /
    max time.  `device` is where the reduction tensors live ("cuda" under
    NCCL, "cpu" under gloo)."""
    edges_all = edges_rank
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        te = torch.tensor([edges_rank], device=device, dtype=torch.float64)
        dist.all_reduce(te)
        edges_all = float(te.item())
    return t_ms, edges_all, edges_all / (t_ms / 1e3) / 1e9


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_launches(trace):
    """Kernels one query launches: set-up (prepare, init), one per step of the
    trace except the levels that ran inside one persistent small-list launch
    (trace mode 4; one launch per run of such levels), and the overflow check."""
    modes = [int(m) for m in trace["mode"]]
    small_runs = sum(1 for i, m in enumerate(modes) if m == 4 and (i == 0 or modes[i - 1] != 4))
    return 2 + sum(1 for m in modes if m != 4) + small_runs + 1


def m_reached_torch(out, deg_t):
    import torch
    reached = out != -1
    return int(torch.where(reached, deg_t, 0).sum().item()), int(reached.sum().item())


def cpu_baseline(g, srcs, budget_s):
    """The oracle (single-threaded FIFO BFS / binary-heap Dijkstra) timed on
    host cores over a bounded sample of the same queries."""
    import oracle
    done_e, t_total, used = 0, 0.0, []
    for kind in ("bfs", "sssp"):
        for s in srcs:
            if t_total > budget_s:
                break
            t0 = time.perf_counter()
            if kind == "bfs":
                res, _ = oracle.bfs(g, int(s))
            else:
                res, _ = oracle.dijkstra(g, int(s))
            dt = time.perf_counter() - t0
            done_e += oracle.m_reached(g, res)
            t_total += dt
            used.append(f"{kind}:{int(s)}")
            if kind == "bfs" and len([u for u in used if u.startswith("bfs")]) >= 2:
                break
    return {"value": done_e / t_total / 1e9 if t_total else None, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(used)} queries of the same workload ({', '.join(used)}), {t_total:.1f} s of CPU time",
            "host_cores": os.cpu_count()}


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on this host's cores,
    on the same workload; each step is one BFS + one SSSP query."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    g = gg.rmat(args.scale, args.edge_factor, seed=1)
    srcs = gg.pick_sources(g, args.sources, seed=1)

    def step(i):
        s = int(srcs[i % len(srcs)])
        t0 = time.perf_counter()
        lev, _ = oracle.bfs(g, s)
        d, _ = oracle.dijkstra(g, s)
        dt = time.perf_counter() - t0
        return oracle.m_reached(g, lev) + oracle.m_reached(g, d), dt

    for i in range(args.warmup):
        step(i)
    tot_e, tot_t = 0, 0.0
    for i in range(args.steps):
        e, dt = step(args.warmup + i)
        tot_e += e
        tot_t += dt
    val = tot_e / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "uint32",
            "data": "synthetic", "config": dict(WORKLOAD, reference="CPU oracle, one BFS + one SSSP per step"),
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of one BFS + one SSSP from one source each"},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def small_configs(torch, reps: int = 3):
    """The two smaller R-MAT configurations and the ER23 shape, every
    strategy: R-MAT scale 14 (edge factor 16, BFS from vertex 0), R-MAT scale
    20 (edge factor 16, weights U[1,255], BFS and SSSP from the
    highest-degree vertex) and Erdos-Renyi with 2^23 vertices and 33.55M
    edges (Table II's ER23 shape; BFS and SSSP from a seeded source).  ms per
    query (mean of `reps` warm runs, CUDA events) and GTEPS = m_reached /
    time."""
    import graphgen as gg
    from paper_1711_00231_gb300 import lb
    out = {}
    g20 = gg.rmat(20, 16, seed=1)
    er23 = gg.erdos_renyi(1 << 23, 33554432, seed=1)
    for name, g, src, kinds in (("rmat14_ef16_vertex0", gg.rmat(14, 16, seed=1), 0, ("bfs",)),
                                ("rmat20_ef16_maxdeg", g20, gg.max_degree_vertex(g20), ("bfs", "sssp")),
                                ("er23_33m_uniform", er23, int(gg.pick_sources(er23, 1, seed=1)[0]), ("bfs", "sssp"))):
        G = lb.Graph.from_csr(g)
        buf = torch.empty(g.n, dtype=torch.int32, device="cuda")
        deg = np.diff(g.offsets)
        row = {"n": g.n, "m": g.m, "source": int(src)}
        for kind in kinds:
            f = G.bfs_dev if kind == "bfs" else G.sssp_dev
            for label in ("BS", "EP", "WD", "NS", "NS_binned", "HP", "HP_binned", "NS_PHYS"):
                s_name = label.replace("_binned", "")
                G.set_options(hp_mode=1 if label == "HP_binned" else 0, ns_mode=1 if label == "NS_binned" else 0)
                f(int(src), s_name, buf)
                torch.cuda.synchronize()
                res = buf.cpu().numpy()
                reached = res >= 0 if kind == "bfs" else res.view(np.uint32) != 0xFFFFFFFF
                m_r = int(deg[reached].sum())
                tot = 0.0
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    f(int(src), s_name, buf)
                    b.record()
                    torch.cuda.synchronize()
                    tot += a.elapsed_time(b)
                ms = tot / reps
                row[f"{kind}_{label}"] = {"ms": ms, "gteps": m_r / (ms / 1e3) / 1e9}
        G.close()
        out[name] = row
    return out


def chunking_ablation(torch, sources: int = 4):
    """The paper's Sec. IV-D experiment on an rmat20-shaped graph (R-MAT
    scale 20, edge factor 16): EP with work chunking (one reservation for all
    edges of the nodes a warp updated) against EP with one atomic per pushed
    edge."""
    import graphgen as gg
    from paper_1711_00231_gb300 import lb
    g = gg.rmat(20, 16, seed=1)
    G = lb.Graph.from_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    srcs = gg.pick_sources(g, sources, seed=1)
    row = {}
    for kind in ("bfs", "sssp"):
        for s_name in ("EP", "EP_NOCHUNK"):
            tot = 0.0
            for s in srcs:
                for rep in range(2):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    (G.bfs_dev if kind == "bfs" else G.sssp_dev)(int(s), s_name, out)
                    b.record()
                    torch.cuda.synchronize()
                    if rep == 1:
                        tot += a.elapsed_time(b)
            row[f"{kind}_{s_name}_ms"] = tot / len(srcs)
        row[f"{kind}_chunking_speedup"] = row[f"{kind}_EP_NOCHUNK_ms"] / row[f"{kind}_EP_ms"]
    G.close()
    row["graph"] = "R-MAT scale 20, edge factor 16, seed 1 (paper: 1.11-3.125x, mean 1.82x on its graphs)"
    return row


def grid_bench(torch):
    """The high-diameter configuration: SSSP (and BFS) from a corner of a
    4096 x 4096 grid (weights U[1,1000]): thousands of small iterations, so
    per-iteration overhead dominates.  Single-query device loop vs the same
    query through the persistent engine."""
    import graphgen as gg
    from paper_1711_00231_gb300 import lb
    from paper_1711_00231_gb300 import serve as sv
    g = gg.grid(4096, 4096, seed=1)
    G = lb.Graph.from_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    row = {"graph": "4096 x 4096 grid, 4-neighbour, weights U[1,1000], source = corner"}
    for kind in ("bfs", "sssp"):
        (G.bfs_dev if kind == "bfs" else G.sssp_dev)(0, "WD", out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        (G.bfs_dev if kind == "bfs" else G.sssp_dev)(0, "WD", out)
        b.record()
        torch.cuda.synchronize()
        st = G.stats()
        row[f"{kind}_ms"] = a.elapsed_time(b)
        row[f"{kind}_iterations"] = st["iterations"]
        row[f"{kind}_us_per_iteration"] = 1e3 * a.elapsed_time(b) / max(1, st["iterations"])
        row[f"{kind}_gteps"] = g.m / (a.elapsed_time(b) / 1e3) / 1e9
        row[f"{kind}_edges_relaxed"] = st["edges_relaxed"]
        row[f"{kind}_work_inflation"] = st["edges_relaxed"] / g.m
        row[f"{kind}_edges_per_iteration"] = st["edges_relaxed"] / max(1, st["iterations"])
    S = sv.Server([G], slots=4)
    for kind in ("bfs", "sssp"):
        S.run_batch([sv.Request(0.0, 0, 0, kind)], [out])
        t0 = time.perf_counter()
        S.run_batch([sv.Request(0.0, 0, 0, kind)], [out])
        row[f"{kind}_server_ms"] = 1e3 * (time.perf_counter() - t0)
    S.close()
    G.close()
    return row


def serving_mix(seed: int = 1):
    """The resident graph mix of the serving workload: 24 R-MAT graphs
    (scale 12..20, edge factor 8/16/32, drawn with `seed`) and 8 grids
    (256^2 .. 2048^2, two weight seeds each), all with weights U[1,255]."""
    import graphgen as gg
    rng = np.random.default_rng(seed)
    scales = rng.integers(12, 21, 24)
    efs = rng.choice([8, 16, 32], 24)
    graphs = [gg.rmat(int(sc), int(ef), seed=100 + i) for i, (sc, ef) in enumerate(zip(scales, efs))]
    for i, side in enumerate([256, 512, 1024, 2048]):
        for ws in (1, 2):
            graphs.append(gg.grid(side, side, seed=200 + 2 * i + ws, weights=(1, 255)))
    return graphs


def serving_bench(args, torch):
    """Batched serving vs one query at a time on the same GPU: 1,024 queries
    (BFS / SSSP 50/50, graph uniform, source uniform over out-degree > 0)
    over 32 resident graphs.  Reports queries/s with every query available at
    once, and p50 / p99 arrival-to-result latency under Poisson arrivals at
    0.8x the one-at-a-time capacity; checks every batched result against the
    one-at-a-time result bit for bit."""
    import graphgen as gg
    from paper_1711_00231_gb300 import lb
    from paper_1711_00231_gb300 import serve as sv
    t0 = time.time()
    cg = serving_mix(1)
    t_gen = time.time() - t0
    G = [lb.Graph.from_csr(g) for g in cg]
    cand = [np.flatnonzero(g.degrees() > 0).astype(np.int32) for g in cg]
    burst = sv.poisson_schedule(args.serve_queries, float("inf"), [g.n for g in cg], cand, seed=1)

    def buffers(reqs):
        # one output per request, sized for that request's graph
        return [torch.empty(cg[r.graph].n, dtype=torch.int32, device="cuda") for r in reqs]

    outs_a, outs_b = buffers(burst), buffers(burst)
    # one at a time: warm every graph's loop, then the whole burst back to back
    for gi, g in enumerate(G):
        tmp = torch.empty(cg[gi].n, dtype=torch.int32, device="cuda")
        g.bfs_dev(int(cand[gi][0]), "WD", tmp)
        g.sssp_dev(int(cand[gi][0]), "WD", tmp)
    torch.cuda.synchronize()
    one = sv.serve_one_at_a_time(G, burst, outs_a)
    # the serving autotuner picks edges per lane, CTAs per SM, tile size and
    # claiming policy on a sample of the burst (its first 64 requests)
    t0 = time.time()
    sample = [(r.graph, r.src, sv.KIND[r.kind]) for r in burst[:64]]
    tuned, tuned_qps = lb.lb_server_autotune([g.h for g in G], sample)
    tune = {"options": {k: tuned[k] for k in ("items", "ctas_per_sm", "tile", "policy")}, "sample_qps": tuned_qps,
            "sample": "first 64 requests of the burst", "seconds": time.time() - t0}
    S = sv.Server(G, ctas_per_sm=tuned["ctas_per_sm"], tile=tuned["tile"], policy=tuned["policy"],
                  items=tuned["items"])
    try:
        res = _serving_runs(args, torch, sv, cg, G, S, cand, burst, outs_a, outs_b, buffers, one, t_gen, tuned)
        res["autotune"] = tune
        return res
    finally:
        S.close()
        for g in G:
            g.close()


def _serving_runs(args, torch, sv, cg, G, S, cand, burst, outs_a, outs_b, buffers, one, t_gen, tuned):
    info = S.info()
    S.run_batch(burst[:64], outs_b[:64])     # warm the persistent kernel
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st = S.run_batch(burst, outs_b)
    torch.cuda.synchronize()
    batched_s = time.perf_counter() - t1
    exact = all(torch.equal(a, b) for a, b in zip(outs_a, outs_b)) and all(x == 0 for x in st)
    rate = 0.8 * one["qps"]
    pois = sv.poisson_schedule(args.serve_queries, rate, [g.n for g in cg], cand, seed=1)
    outs_a, outs_b = buffers(pois), buffers(pois)
    one_p = sv.serve_one_at_a_time(G, pois, outs_a)
    srv_p = sv.serve(S, pois, outs_b, timeout_s=args.serve_timeout)
    torch.cuda.synchronize()
    exact_p = all(torch.equal(a, b) for a, b in zip(outs_a, outs_b)) and srv_p["statuses_ok"]
    # the same arrivals with the other claiming policy
    other = 1 - tuned["policy"]
    S_rr = sv.Server(G, ctas_per_sm=tuned["ctas_per_sm"], tile=tuned["tile"], policy=other, items=tuned["items"])
    try:
        outs_c = buffers(pois)
        S_rr.run_batch(burst[:64], buffers(burst[:64]))
        srv_rr = sv.serve(S_rr, pois, outs_c, timeout_s=args.serve_timeout)
        torch.cuda.synchronize()
        exact_p = exact_p and all(torch.equal(a, c) for a, c in zip(outs_a, outs_c)) and srv_rr["statuses_ok"]
    finally:
        S_rr.close()
    rate_hi = 0.8 * args.serve_queries / batched_s
    pois_hi = sv.poisson_schedule(args.serve_queries, rate_hi, [g.n for g in cg], cand, seed=2)
    outs_b = buffers(pois_hi)
    srv_hi = sv.serve(S, pois_hi, outs_b, timeout_s=args.serve_timeout)
    info2 = S.info()
    # results of the high-rate run against the single-query calls (untimed)
    outs_a = buffers(pois_hi)
    for r, o in zip(pois_hi, outs_a):
        (G[r.graph].bfs_dev if r.kind == "bfs" else G[r.graph].sssp_dev)(r.src, "WD", o)
    torch.cuda.synchronize()
    exact_hi = all(torch.equal(a, b) for a, b in zip(outs_a, outs_b)) and srv_hi["statuses_ok"]
    return {"workload": "32 graphs (24 R-MAT scale 12-20 ef 8/16/32, 8 grids 256^2-2048^2), weights U[1,255]; "
                        f"{args.serve_queries} queries, BFS/SSSP 50/50, seed 1",
            "one_at_a_time_qps": one["qps"], "batched_qps": args.serve_queries / batched_s,
            "speedup_qps": (args.serve_queries / batched_s) / one["qps"],
            "poisson_rate_qps": rate,
            "one_at_a_time_latency": {k: one_p[k] for k in ("p50_ms", "p99_ms", "mean_ms")},
            "batched_latency": {k: srv_p[k] for k in ("p50_ms", "p99_ms", "mean_ms")},
            f"batched_latency_policy{other}": {k: srv_rr[k] for k in ("p50_ms", "p99_ms", "mean_ms")},
            "claiming": f"policy {tuned['policy']} (0: oldest query first, then round robin; 1: round robin only); "
                        f"policy {other} beside it with the other options unchanged",
            "pool_bytes": info["pool_bytes"], "query_bytes_largest_graph": info["slot_bytes"],
            "batched_latency_at_0.8x_batched_capacity": {"rate_qps": rate_hi, **{k: srv_hi[k] for k in
                                                                                 ("p50_ms", "p99_ms", "qps")}},
            "exact_vs_one_at_a_time": bool(exact and exact_p and exact_hi), "slots": info["slots"],
            "grid": info["grid"],
            "kernel_launches": info2["kernel_launches"], "generate_s": t_gen}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serve_only:
        import torch
        from paper_1711_00231_gb300 import _build
        _build.build()
        print(json.dumps({"batched": serving_bench(args, torch)}), flush=True)
        return
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import graphgen as gg
    from paper_1711_00231_gb300 import _build, lb
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()

    t0 = time.time()
    g = gg.rmat(args.scale, args.edge_factor, seed=1)
    t_gen = time.time() - t0
    srcs = rank_sources(g, args.sources, rank, world)
    t0 = time.time()
    G = lb.Graph.from_csr(g)
    if args.loop_mode:
        G.set_options(loop_mode=args.loop_mode)
    if args.wd_tile:
        G.set_options(wd_tile=args.wd_tile)
    if args.hp_mode:
        G.set_options(hp_mode=args.hp_mode)
    if args.ns_mode:
        G.set_options(ns_mode=args.ns_mode)
    t_upload = time.time() - t0
    kinds = tuple(k for k in args.kinds.split(",") if k)
    strat = args.strategy
    # the library's autotuner picks the options (tile size, CTAs per SM,
    # bin thresholds, granule size, ... for the strategy) on two sources of
    # a separate draw; the timed queries run with what it chose
    tune = None
    if not args.no_tune and not args.wd_tile:
        t0 = time.time()
        tsrc = gg.pick_sources(g, 2, seed=2)
        best, best_ms = G.autotune("both" if len(kinds) == 2 else kinds[0], strat, tsrc)
        tune = {"options": best, "ms_per_source": best_ms, "sources": [int(s) for s in tsrc],
                "seconds": time.time() - t0}
    run_opts = G.options()
    deg_t = torch.from_numpy(np.diff(g.offsets)).cuda()
    stream = torch.cuda.current_stream()
    n = g.n
    out = torch.empty(n, dtype=torch.int32, device="cuda")

    def query(kind, s, strategy=strat):
        if kind == "bfs":
            G.bfs_dev(int(s), strategy, out, None, stream)
        else:
            G.sssp_dev(int(s), strategy, out, None, stream)

    # work per query (edges and vertices reached), from a first run
    work = {}
    trace_first = {}
    for kind in kinds:
        for s in srcs:
            query(kind, s)
            torch.cuda.synchronize()
            st = G.stats()
            if st["status"] != 0:
                raise SystemExit(f"query failed: {kind} src={s} status={st['status']}")
            work[(kind, int(s))] = m_reached_torch(out, deg_t) + (kernel_launches(G.trace()), st["iterations"],
                                                                  st["edges_relaxed"])

    ev = {k: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
          for k in kinds}

    def step(record=False):
        for kind in kinds:
            for i, s in enumerate(srcs):
                if record:
                    ev[kind][i][0].record(stream)
                query(kind, s)
                if record:
                    ev[kind][i][1].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    per_query_ms = {k: np.zeros(len(srcs)) for k in kinds}
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step(record=True)
        torch.cuda.synchronize()
        for kind in kinds:
            for i in range(len(srcs)):
                per_query_ms[kind][i] += ev[kind][i][0].elapsed_time(ev[kind][i][1])
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    elapsed_ms = start.elapsed_time(stop)
    # per-step device times of one warm query of each kind (from the trace)
    for kind in kinds:
        query(kind, srcs[0])
        torch.cuda.synchronize()
        prev = 0
        steps_first = []
        for rec in G.trace():
            steps_first.append({"level": int(rec["level"]), "list": int(rec["list_size"]),
                                "edges": int(rec["edges"]), "us": round((int(rec["t_ns"]) - prev) / 1e3, 1)})
            prev = int(rec["t_ns"])
        trace_first[kind] = steps_first
    # device time of the queries themselves (the host sync between steps excluded)
    dev_ms = float(sum(per_query_ms[k].sum() for k in kinds))
    edges_rank = sum(work[(k, int(s))][0] for k in kinds for s in srcs) * args.steps
    t_ms, edges_all, value = combine_ranks(dev_ms, edges_rank, world, "cuda")

    res = {}
    for kind in kinds:
        e = sum(work[(kind, int(s))][0] for s in srcs) * args.steps
        v = sum(work[(kind, int(s))][1] for s in srcs) * args.steps
        t = per_query_ms[kind].sum() / 1e3
        be, bv = BYTES[kind]
        res[kind] = {"gteps": e / t / 1e9, "ms_per_query": 1e3 * t / (args.steps * len(srcs)),
                     "algorithmic_gbs": (be * e + bv * v) / t / 1e9,
                     "launches": sum(work[(kind, int(s))][2] for s in srcs) * args.steps,
                     "iterations_mean": float(np.mean([work[(kind, int(s))][3] for s in srcs])),
                     "work_inflation": sum(work[(kind, int(s))][4] for s in srcs) / max(
                         1, sum(work[(kind, int(s))][0] for s in srcs))}
    peak, peak_kind = measured_peak()
    dom = max(kinds, key=lambda k: per_query_ms[k].sum())
    achieved = res[dom]["algorithmic_gbs"]
    def roof(kind):
        a = res[kind]["algorithmic_gbs"]
        return {"bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                "traffic": None,
                "traffic_note": "captured at R-MAT scale 22 only (profiles/k_step_wd_traffic_rmat22_ef32.md: BFS "
                                "0.65x, SSSP 1.72x the algorithmic bytes per query); not scaled, since at scale 24 "
                                "the distance array no longer fits in L2 and traffic does not grow in proportion",
                "kernel": f"k_step_wd ({kind})", "peak_source": f"{peak_kind} hbm_gbs",
                "unit_of_work": "one query (all its relax launches + set-up); algorithmic bytes per query "
                                f"= {BYTES[kind][0]} B x m_reached + {BYTES[kind][1]} B x n_reached"}
    roofline = roof(dom)
    roofline_by_kind = {k: roof(k) for k in kinds}

    extra = {}
    if rank == 0 and not args.no_compare:
        cmp_src = srcs[:args.compare_sources]
        for kind in kinds:
            row = {}
            # every strategy's result is compared with WD's, element by element
            # (WD itself equals the oracle in the GPU tests on this workload)
            wd_ref = {}
            for s in cmp_src:
                query(kind, s, "WD")
                wd_ref[int(s)] = out.clone()
            for label in ("BS", "EP", "WD", "NS", "NS_binned", "HP", "HP_binned", "NS_PHYS"):
                # *_binned: HP with hp_mode 1 (degree-binned sub-worklists in one
                # step), NS with ns_mode 1 (granules by a thread, a warp or the CTA)
                s_name = label.replace("_binned", "")
                G.set_options(hp_mode=1 if label == "HP_binned" else 0, ns_mode=1 if label == "NS_binned" else 0)
                tot = 0.0
                e_tot = 0
                b_tot = 0
                per_q = []
                exact = True
                for s in cmp_src:
                    query(kind, s, s_name)   # warm (builds its workspace / loop)
                    torch.cuda.synchronize()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    query(kind, s, s_name)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b)
                    tot += ms
                    m_r, n_r = work[(kind, int(s))][0], work[(kind, int(s))][1]
                    e_tot += m_r
                    b_tot += BYTES[kind][0] * m_r + BYTES[kind][1] * n_r
                    per_q.append(m_r / (ms / 1e3) / 1e9)
                    exact = exact and G.stats()["status"] == 0 and bool(torch.equal(out, wd_ref[int(s)]))
                alg = b_tot / (tot / 1e3) / 1e9
                mem = G.mem_report(s_name)
                row[label] = {"ms_per_query": tot / len(cmp_src), "gteps": e_tot / (tot / 1e3) / 1e9,
                              "gteps_mean": float(np.mean(per_q)),
                              "gteps_hmean": float(len(per_q) / sum(1.0 / x for x in per_q)),
                              "gteps_min": float(min(per_q)), "algorithmic_gbs": alg, "hbm_frac": alg / peak,
                              "extra_device_bytes": int(mem["extra_total"]), "exact_vs_wd": exact}
            del wd_ref
            G.set_options(hp_mode=0, ns_mode=0)
            row["speedup_wd_vs_bs"] = row["BS"]["ms_per_query"] / row["WD"]["ms_per_query"]
            row["speedup_wd_vs_ep"] = row["EP"]["ms_per_query"] / row["WD"]["ms_per_query"]
            extra[kind] = row
        G.release()
        extra["chunking_ablation"] = chunking_ablation(torch)
        extra["configs"] = small_configs(torch)
        extra["grid4096"] = grid_bench(torch)

    # end to end through the host-buffer C-ABI calls: every result is copied
    # into pinned host memory inside the timed region.  The batched calls
    # (lb_bfs_batch / lb_sssp_batch: one call per kind over all sources)
    # copy query i's result while query i + 1 runs; the one-query calls
    # (lb_bfs / lb_sssp) are timed beside them
    e2e = None
    if rank == 0:
        host = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
        hostu = host.view(np.uint32)
        hb_t = torch.empty(len(srcs) * n, dtype=torch.int32, pin_memory=True)
        hb = hb_t.numpy()
        hbu = hb.view(np.uint32)
        src_list = [int(s) for s in srcs]
        # warm both kinds (the comparison above released the workspaces, so
        # each kind's workspace and device loop are rebuilt here, outside
        # the timed region), the second result buffer and the copy stream
        for kind in kinds:
            if kind == "bfs":
                G.bfs(src_list[0], strat)
                lb.lb_bfs_batch(G.h, src_list[:2], strat, hb[:2 * n])
            else:
                G.sssp(src_list[0], strat)
                lb.lb_sssp_batch(G.h, src_list[:2], strat, hbu[:2 * n])
        e_done = sum(work[(kind, s)][0] for kind in kinds for s in src_list)
        t0 = time.perf_counter()
        for kind in kinds:
            if kind == "bfs":
                lb.lb_bfs_batch(G.h, src_list, strat, hb)
            else:
                lb.lb_sssp_batch(G.h, src_list, strat, hbu)
        dt = time.perf_counter() - t0
        t0 = time.perf_counter()
        for kind in kinds:
            for s in src_list:
                if kind == "bfs":
                    lb.lb_bfs(G.h, s, strat, host)
                else:
                    lb.lb_sssp(G.h, s, strat, hostu)
        dt1 = time.perf_counter() - t0
        e2e = {"value": e_done / dt / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(srcs) * len(kinds),
               "d2h_bytes_per_step": 4 * n * len(srcs) * len(kinds),
               "call": "lb_bfs_batch / lb_sssp_batch (all sources of a kind in one call)",
               "one_query_calls": {"value": e_done / dt1 / 1e9, "unit": "GTEPS", "call": "lb_bfs / lb_sssp"},
               "note": "graph resident; the source ids go in as host arguments and every n x 4 B result comes "
                       "back to pinned host memory (host-timed, wall clock)"}
        del hb, hbu, hb_t

    batched = None
    if rank == 0 and not args.no_serve:
        try:
            batched = serving_bench(args, torch)
        except Exception as ex:  # the kernel-only line still prints; the failure is reported in it
            batched = {"error": f"{type(ex).__name__}: {ex}"[:4000]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(g, srcs[:2], args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "uint32", "data": "synthetic",
                "config": dict(WORKLOAD, strategy=strat, parallelism=f"replicas{world}", n=g.n, m=g.m,
                               scale=args.scale, edge_factor=args.edge_factor, sources=len(srcs), kinds=list(kinds),
                               loop="device (CUDA graph WHILE)" if args.loop_mode == 0 else "host",
                               options=run_opts, autotune=tune),
                "roofline": roofline, "roofline_by_kind": roofline_by_kind, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks,
                "gpu_launches": sum(res[k]["launches"] for k in kinds),
                "per_kind": res, "strategies": extra, "batched": batched,
                "steps_of_first_query": trace_first,
                "setup_s": {"generate": t_gen, "upload": t_upload}, "elapsed_ms_timed_region": elapsed_ms}
        print(json.dumps(line), flush=True)
    G.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
