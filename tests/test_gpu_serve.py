"""Batched / served queries through the persistent multi-query engine
(lb_server_*): every result must equal the oracle's bit for bit, alone and
in a mix, whatever the arrival pattern, slot count or tile size."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1711_00231_gb300 import lb
from paper_1711_00231_gb300 import serve as sv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_00231_gb300 import _build
    _build.build()


@pytest.fixture(scope="module")
def mix():
    graphs = [gg.rmat(12, 8, seed=1), gg.rmat(14, 16, seed=2), gg.grid(64, 48, seed=3),
              gg.erdos_renyi(3000, 12000, seed=4), gg.rmat(13, 32, seed=5, weights=None),
              gg.from_edges(6, [0, 1, 2], [1, 2, 3], [1, 2, 3])]
    handles = [lb.Graph.from_csr(g) for g in graphs]
    yield graphs, handles
    for h in handles:
        h.close()


def reference(g, kind, src):
    if kind == "bfs":
        return oracle.bfs(g, src)[0]
    return oracle.dijkstra(g, src)[0].view(np.int32)


def make_requests(graphs, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        gi = int(rng.integers(0, len(graphs)))
        kind = "sssp" if graphs[gi].weights is not None and rng.random() < 0.5 else "bfs"
        reqs.append(sv.Request(0.0, gi, int(rng.integers(0, graphs[gi].n)), kind))
    return reqs


@pytest.mark.parametrize("slots,tile,policy", [(0, 0, 0), (3, 256, 0), (17, 8192, 0), (0, 0, 1), (5, 1024, 1)])
def test_batch_matches_oracle(mix, slots, tile, policy):
    # policy 0: the oldest query's tiles first; 1: round robin only
    import torch
    graphs, handles = mix
    reqs = make_requests(graphs, 60, seed=slots + tile)
    outs = [torch.full((graphs[r.graph].n,), 7, dtype=torch.int32, device="cuda") for r in reqs]
    S = sv.Server(handles, slots=slots, tile=tile, policy=policy)
    try:
        st = S.run_batch(reqs, outs, timeout_s=120)
        assert all(x == 0 for x in st), st
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src)), r
        info = S.info()
        assert info["completed"] == len(reqs) and info["slots"] >= 1
        if slots:
            assert info["slots"] == slots
    finally:
        S.close()


def test_same_result_alone_and_in_the_mix(mix):
    import torch
    graphs, handles = mix
    S = sv.Server(handles, slots=8)
    try:
        probe = sv.Request(0.0, 1, 77, "sssp")
        alone = torch.empty(graphs[1].n, dtype=torch.int32, device="cuda")
        assert S.run_batch([probe], [alone]) == [0]
        reqs = make_requests(graphs, 40, seed=9)
        reqs.insert(17, probe)
        outs = [torch.empty(graphs[r.graph].n, dtype=torch.int32, device="cuda") for r in reqs]
        assert all(x == 0 for x in S.run_batch(reqs, outs))
        torch.cuda.synchronize()
        assert torch.equal(outs[17], alone)
        # and equal to the single-query entry point
        single = torch.empty_like(alone)
        handles[1].sssp_dev(77, "WD", single)
        torch.cuda.synchronize()
        assert torch.equal(single, alone)
    finally:
        S.close()


def test_continuous_arrivals_and_relaunch(mix):
    import torch
    graphs, handles = mix
    S = sv.Server(handles, slots=4, idle_us=200)
    try:
        reqs = make_requests(graphs, 30, seed=11)
        for i, r in enumerate(reqs):
            r.arrival_s = 0.002 * i
        outs = [torch.empty(graphs[r.graph].n, dtype=torch.int32, device="cuda") for r in reqs]
        res = sv.serve(S, reqs, outs, timeout_s=120)
        assert res["statuses_ok"] and res["queries"] == 30
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src))
        time.sleep(0.05)      # longer than idle_us: the persistent kernel leaves
        more = make_requests(graphs, 5, seed=12)
        outs2 = [torch.empty(graphs[r.graph].n, dtype=torch.int32, device="cuda") for r in more]
        assert all(x == 0 for x in S.run_batch(more, outs2))
        torch.cuda.synchronize()
        for r, o in zip(more, outs2):
            assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src))
        assert S.info()["kernel_launches"] >= 2
    finally:
        S.close()


def test_many_small_rounds_with_few_slots(mix):
    # two slots, a short idle timeout and a steady trickle: the persistent
    # kernel keeps finding no work between requests, leaves, and is
    # relaunched many times; every result must still be exact
    import torch
    graphs, handles = mix
    S = sv.Server(handles, slots=2, idle_us=50, tile=256)
    try:
        reqs = make_requests(graphs, 120, seed=21)
        for i, r in enumerate(reqs):
            r.arrival_s = 0.0005 * i
        outs = [torch.empty(graphs[r.graph].n, dtype=torch.int32, device="cuda") for r in reqs]
        res = sv.serve(S, reqs, outs, timeout_s=120)
        assert res["statuses_ok"]
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src))
    finally:
        S.close()


def test_many_jobs_in_flight(mix):
    # many slots busy at once with small tiles: jobs open and close on every
    # slot while hundreds of CTAs scan and claim, so a claim taken against a
    # job that has just been replaced is common; every result must be exact
    import torch
    graphs, handles = mix
    S = sv.Server(handles, slots=96, tile=256)
    try:
        for rep in range(2):
            reqs = make_requests(graphs, 400, seed=31 + rep)
            outs = [torch.empty(graphs[r.graph].n, dtype=torch.int32, device="cuda") for r in reqs]
            st = S.run_batch(reqs, outs, timeout_s=120)
            assert all(x == 0 for x in st), st
            torch.cuda.synchronize()
            for r, o in zip(reqs, outs):
                assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src)), r
        state = S.state()
        assert state["busy_slots"] == 0 and state["active"] == 0 and state["completed"] == 800
    finally:
        S.close()


def test_queries_continue_across_launch_time_limits():
    # a 2 ms launch limit: grid queries of thousands of iterations (tens of
    # ms) outlive many launches, and each relaunch continues them from the
    # state the slots keep in device memory; the results must still be exact
    import torch
    g = gg.grid(1024, 1024, seed=5)
    G = lb.Graph.from_csr(g)
    S = sv.Server([G], slots=4, launch_ms=2)
    try:
        reqs = [sv.Request(0.0, 0, 0, "sssp"), sv.Request(0.0, 0, g.n - 1, "sssp"), sv.Request(0.0, 0, 7, "bfs"),
                sv.Request(0.0, 0, g.n // 2, "sssp")]
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in reqs]
        st = S.run_batch(reqs, outs, timeout_s=120)
        assert all(x == 0 for x in st), st
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), reference(g, r.kind, r.src)), r
        assert S.info()["kernel_launches"] >= 3
    finally:
        S.close()
        G.close()


def test_overflow_and_invalid_requests(mix):
    import torch
    graphs, handles = mix
    big = 0x80000000
    g = gg.from_edges(4, [0, 1, 2], [1, 2, 3], [big, big - 3, 5])
    G = lb.Graph.from_csr(g)
    S = sv.Server([G, handles[4]], slots=2)
    try:
        out = torch.empty(4, dtype=torch.int32, device="cuda")
        st = S.run_batch([sv.Request(0.0, 0, 0, "sssp")], [out])
        assert st == [lb.LB_ERR_OVERFLOW]
        assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.dijkstra(g, 0)[0])
        with pytest.raises(lb.LbError):
            S.submit(0, 9, "bfs", out)            # source out of range
        out1 = torch.empty(graphs[4].n, dtype=torch.int32, device="cuda")
        with pytest.raises(lb.LbError):
            S.submit(1, 0, "sssp", out1)          # unweighted graph
        with pytest.raises(lb.LbError):
            S.submit(5, 0, "bfs", out)            # no such graph
        with pytest.raises(ValueError):
            S.submit(1, 0, "bfs", out)            # output smaller than the graph
    finally:
        S.close()
        G.close()


def test_admission_by_memory_queues_what_does_not_fit():
    # a pool that holds about two workspaces of the large graph: queries
    # on it wait (pending) until completions return memory, the small
    # graph's queries fill the rest, every result is exact and the whole
    # pool is free at the end
    import torch
    big = gg.grid(512, 512, seed=6)
    small = gg.rmat(11, 8, seed=7)
    graphs = [big, small]
    handles = [lb.Graph.from_csr(g) for g in graphs]
    try:
        probe = sv.Server(handles)
        ws_big = probe.info()["slot_bytes"]
        probe.close()
        free, _ = torch.cuda.mem_get_info()
        S = sv.Server(handles, slots=64, mem_fraction=2.5 * ws_big / free)
        try:
            info = S.info()
            assert 2 * ws_big <= info["pool_bytes"] < 3 * ws_big
            rng = np.random.default_rng(3)
            reqs = [sv.Request(0.0, i % 2, int(rng.integers(0, graphs[i % 2].n)), "sssp" if i % 3 else "bfs")
                    for i in range(24)]
            outs = [torch.full((graphs[r.graph].n,), 7, dtype=torch.int32, device="cuda") for r in reqs]
            tick = {S.submit(r.graph, r.src, r.kind, o): i for i, (r, o) in enumerate(zip(reqs, outs))}
            saw_pending = S.info()["pending"] > 0
            left, t_end = len(reqs), time.perf_counter() + 120
            while left:
                for c in S.poll():
                    assert c[1] == 0
                    tick.pop(c[0])
                    left -= 1
                inf = S.info()
                saw_pending = saw_pending or inf["pending"] > 0
                assert 0 <= inf["pool_free"] <= inf["pool_bytes"]
                assert time.perf_counter() < t_end, S.state()
            assert saw_pending
            info = S.info()
            assert info["pool_free"] == info["pool_bytes"] and info["pending"] == 0
            torch.cuda.synchronize()
            for r, o in zip(reqs, outs):
                assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src)), r
        finally:
            S.close()
    finally:
        for h in handles:
            h.close()


def test_server_autotune_picks_grid_options(mix):
    # the serving autotuner runs a sample batch under each candidate of its
    # grid and returns the fastest; a server built with it gives exact results
    import torch
    graphs, handles = mix
    reqs = make_requests(graphs, 24, seed=21)
    sample = [(r.graph, r.src, sv.KIND[r.kind]) for r in reqs]
    best, qps = lb.lb_server_autotune([h.h for h in handles], sample, slots=16)
    assert qps > 0
    assert best["items"] in (2, 3) and best["ctas_per_sm"] in (0, 3) and best["tile"] in (4096, 8192)
    assert best["policy"] in (0, 1) and best["slots"] == 16
    S = sv.Server(handles, slots=best["slots"], ctas_per_sm=best["ctas_per_sm"], tile=best["tile"],
                  policy=best["policy"], items=best["items"])
    try:
        outs = [torch.full((graphs[r.graph].n,), 7, dtype=torch.int32, device="cuda") for r in reqs]
        assert all(x == 0 for x in S.run_batch(reqs, outs, timeout_s=120))
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            assert np.array_equal(o.cpu().numpy(), reference(graphs[r.graph], r.kind, r.src)), r
    finally:
        S.close()
    with pytest.raises(lb.LbError) as ei:
        lb.lb_server_autotune([h.h for h in handles], [(0, graphs[0].n, 0)])
    assert ei.value.status == lb.LB_ERR_ARG
