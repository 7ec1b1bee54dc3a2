"""Request loop for serving BFS / SSSP queries over resident graphs.

``Server`` wraps the library's persistent multi-query engine
(lb_server_*): requests are submitted as they arrive and completions are
polled, so queries that arrive while others run are admitted as soon as a
slot is free and their iterations interleave on the GPU (continuous
batching).  ``serve`` replays an arrival schedule against it and records
arrival-to-result latency; ``serve_one_at_a_time`` replays the same
schedule through the single-query calls (lb_bfs_dev / lb_sssp_dev), one
query after another, as the comparison.  All device work runs in the
library's kernels; this module only schedules calls and keeps time.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import lb

KIND = {"bfs": lb.LB_KIND_BFS, "sssp": lb.LB_KIND_SSSP}


@dataclass
class Request:
    arrival_s: float   # offset from the start of the run
    graph: int
    src: int
    kind: str          # "bfs" or "sssp"


class Server:
    def __init__(self, graphs: Sequence["lb.Graph"], slots: int = 0, ctas_per_sm: int = 0, tile: int = 0,
                 idle_us: int = 0, mem_fraction: float = 0.0, launch_ms: int = 0, policy: int = 0, items: int = 0):
        self.graphs = list(graphs)
        self.h = lb.lb_server_create([g.h for g in self.graphs], slots, ctas_per_sm, tile, idle_us, mem_fraction,
                                     launch_ms, policy, items)

    def submit(self, graph: int, src: int, kind: str, out_dev) -> int:
        if 0 <= graph < len(self.graphs):
            lb._need(out_dev, self.graphs[graph].n)
        return lb.lb_server_submit(self.h, graph, src, KIND[kind], out_dev)

    def poll(self):
        return lb.lb_server_poll(self.h)

    def info(self) -> dict:
        return lb.lb_server_info(self.h)

    def stop(self):
        lb.lb_server_stop(self.h)

    def state(self) -> dict:
        return lb.lb_server_state(self.h)

    def close(self):
        if getattr(self, "h", None):
            lb.lb_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_batch(self, reqs: Sequence[Request], outs, timeout_s: float = 600.0):
        """Submits every request at once and waits for all of them."""
        tick = {}
        for i, r in enumerate(reqs):
            tick[self.submit(r.graph, r.src, r.kind, outs[i])] = i
        status = [None] * len(reqs)
        left = len(reqs)
        t_end = time.perf_counter() + timeout_s
        while left:
            for c in self.poll():
                status[tick[c[0]]] = c[1]
                left -= 1
            if left and time.perf_counter() > t_end:
                raise TimeoutError(f"{left} queries still running; engine state {self.state()}")
        return status


def _percentiles(lat: List[float]) -> dict:
    a = np.asarray(lat) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p90_ms": float(np.percentile(a, 90)),
            "p99_ms": float(np.percentile(a, 99)), "mean_ms": float(a.mean()), "max_ms": float(a.max())}


def serve(server: Server, reqs: Sequence[Request], outs, timeout_s: float = 600.0) -> dict:
    """Replays ``reqs`` (sorted by arrival) against the engine.  Latency =
    time from a request's arrival to the poll that returns its result."""
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival_s)
    arrival = np.zeros(len(reqs))
    done_at = np.zeros(len(reqs))
    status = [None] * len(reqs)
    tick = {}
    t0 = time.perf_counter()
    nxt, left = 0, len(reqs)
    while left:
        now = time.perf_counter() - t0
        while nxt < len(order) and reqs[order[nxt]].arrival_s <= now:
            i = order[nxt]
            r = reqs[i]
            arrival[i] = r.arrival_s
            tick[server.submit(r.graph, r.src, r.kind, outs[i])] = i
            nxt += 1
        comp = server.poll()
        if comp:
            tnow = time.perf_counter() - t0
            for c in comp:
                i = tick.pop(c[0])
                done_at[i] = tnow
                status[i] = c[1]
                left -= 1
        if now > timeout_s:
            raise TimeoutError(f"{left} queries unfinished; engine state {server.state()}")
    span = done_at.max() - min(r.arrival_s for r in reqs)
    res = {"queries": len(reqs), "seconds": float(span), "qps": len(reqs) / span,
           "statuses_ok": all(s == 0 for s in status)}
    res.update(_percentiles(list(done_at - arrival)))
    return res


def serve_one_at_a_time(graphs: Sequence["lb.Graph"], reqs: Sequence[Request], outs, strategy: str = "WD",
                        stream=None) -> dict:
    """The same schedule through the single-query calls, one query at a
    time in arrival order (a FIFO queue in front of one GPU)."""
    import torch
    order = sorted(range(len(reqs)), key=lambda i: reqs[i].arrival_s)
    stream = stream or torch.cuda.current_stream()
    arrival = np.zeros(len(reqs))
    done_at = np.zeros(len(reqs))
    t0 = time.perf_counter()
    for i in order:
        r = reqs[i]
        while time.perf_counter() - t0 < r.arrival_s:
            pass
        g = graphs[r.graph]
        if r.kind == "bfs":
            g.bfs_dev(r.src, strategy, outs[i], None, stream)
        else:
            g.sssp_dev(r.src, strategy, outs[i], None, stream)
        stream.synchronize()
        arrival[i] = r.arrival_s
        done_at[i] = time.perf_counter() - t0
    span = done_at.max() - min(r.arrival_s for r in reqs)
    res = {"queries": len(reqs), "seconds": float(span), "qps": len(reqs) / span}
    res.update(_percentiles(list(done_at - arrival)))
    return res


def poisson_schedule(n: int, rate_qps: float, graphs_n: Sequence[int], graphs_src: Sequence[np.ndarray],
                     seed: int = 1, sssp_ok: Optional[Sequence[bool]] = None) -> List[Request]:
    """n requests with exponential inter-arrival times (rate_qps; inf = all
    at t = 0), graph uniform, kind BFS / SSSP 50/50, source uniform among
    the graph's candidate sources."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        if np.isfinite(rate_qps):
            t += rng.exponential(1.0 / rate_qps)
        gi = int(rng.integers(0, len(graphs_n)))
        kind = "sssp" if rng.random() < 0.5 and (sssp_ok is None or sssp_ok[gi]) else "bfs"
        cand = graphs_src[gi]
        src = int(cand[int(rng.integers(0, len(cand)))])
        out.append(Request(t if np.isfinite(rate_qps) else 0.0, gi, src, kind))
    return out
