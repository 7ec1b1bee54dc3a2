"""The autotuner (lb_autotune): for every strategy it must return options
from its candidate grid, keep them on the graph, and leave results exact
(the options choose schedules, never values).  When a candidate fails part
way through (a device allocation refused through the allocator hook), the
caller's options must come back unchanged."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1711_00231_gb300 import lb

pytestmark = pytest.mark.gpu

# the candidate values of each field the grid varies (include/lb.h)
GRID = {
    "WD": {"wd_tile": {2048, 4096, 8192, 16384}, "ctas_per_sm": {0, 2, 3, 4}},
    "HP": {"hp_mode": {0, 1}, "hp_threshold": {256, 1024, 4096}, "hp_depth": {1, 2, 3}},
    "NS": {"ns_mode": {0, 1}, "mdt_override": {0, 32, 256, 2048}},
    "NS_PHYS": {"mdt_override": {0, 32, 256, 2048}},
    "BS": {"ctas_per_sm": {0, 2, 3, 4}},
    "EP": {"ctas_per_sm": {0, 2, 3, 4}},
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_00231_gb300 import _build
    _build.build()


@pytest.mark.parametrize("strategy", list(GRID))
def test_autotune_returns_grid_options_and_exact_results(strategy):
    g = gg.rmat(14, 16, seed=1)
    srcs = [0, gg.max_degree_vertex(g)]
    G = lb.Graph.from_csr(g)
    try:
        G.set_options(loop_mode=0, hist_bins=10)
        best, ms = G.autotune("both", strategy, srcs)
        assert ms > 0
        for field, values in GRID[strategy].items():
            assert best[field] in values, (strategy, field, best[field])
        assert best["bitmap_place"] in range(8)  # the placement pass after the grid
        if strategy == "WD":  # the small-list pass: the default threshold or off
            assert best["small_edges"] in {0, 16384}
        assert G.options() == best
        if strategy == "HP" and best["hp_mode"] == 1:
            assert best["thread_max"] in {8, 32, 128} and best["hp_warp_max"] in {512, 4096}
        if strategy == "NS" and best["ns_mode"] == 1:
            assert best["thread_max"] in {8, 32, 128}
        for src in srcs:
            assert np.array_equal(G.bfs(src, strategy), oracle.bfs(g, src)[0])
            d, rc = G.sssp(src, strategy)
            assert rc == lb.LB_OK and np.array_equal(d, oracle.dijkstra(g, src)[0])
    finally:
        G.close()


def test_autotune_keeps_the_small_list_launch_on_a_grid():
    # a 256 x 256 grid has 511 BFS levels of at most a few hundred edges:
    # the persistent small-list launch (a grid barrier per level) beats a
    # launch per level by far, so the tuner must keep it on
    g = gg.grid(256, 256, seed=1)
    G = lb.Graph.from_csr(g)
    try:
        best, ms = G.autotune("both", "WD", [0])
        assert best["small_edges"] > 0, best
        assert np.array_equal(G.bfs(0, "WD"), oracle.bfs(g, 0)[0])
        d, rc = G.sssp(0, "WD")
        assert rc == lb.LB_OK and np.array_equal(d, oracle.dijkstra(g, 0)[0])
    finally:
        G.close()


def test_autotune_single_kind_and_argument_errors():
    g = gg.rmat(12, 8, seed=3)
    G = lb.Graph.from_csr(g)
    try:
        best, ms = G.autotune("bfs", "WD", [1])
        assert ms > 0 and best["wd_tile"] in GRID["WD"]["wd_tile"]
        with pytest.raises(lb.LbError) as ei:
            G.autotune("bfs", "WD", [g.n])
        assert ei.value.status == lb.LB_ERR_ARG
    finally:
        G.close()
    gu = gg.rmat(10, 8, seed=3, weights=None)
    G = lb.Graph.from_csr(gu)
    try:
        with pytest.raises(lb.LbError) as ei:
            G.autotune("both", "WD", [0])
        assert ei.value.status == lb.LB_ERR_UNSUPPORTED
    finally:
        G.close()


class Hook:
    """Device allocator backed by torch tensors that can be told to refuse."""

    def __init__(self):
        self.keep = {}
        self.refuse = False

    def alloc(self, size):
        import torch
        if self.refuse:
            return 0
        t = torch.empty(max(size, 1), dtype=torch.uint8, device="cuda")
        self.keep[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr):
        self.keep.pop(ptr, None)


def test_autotune_restores_options_after_a_failed_candidate():
    # NS_PHYS candidates rebuild the split map for each granule size; with
    # allocations refused the first candidate fails, and the options set
    # before the call must be in force again
    g = gg.rmat(12, 8, seed=2)
    h = Hook()
    lb.lb_set_allocator(h.alloc, h.free)
    try:
        G = lb.Graph.from_csr(g)
        try:
            G.set_options(wd_tile=4096, ctas_per_sm=2, thread_max=16, mdt_override=7, hp_depth=2)
            before = G.options()
            G.bfs(0, "WD")
            h.refuse = True
            with pytest.raises(lb.LbError) as ei:
                G.autotune("both", "NS_PHYS", [0, 1])
            assert ei.value.status == lb.LB_ERR_OOM
            assert G.options() == before
            h.refuse = False
            assert np.array_equal(G.bfs(0, "NS_PHYS"), oracle.bfs(g, 0)[0])
            assert G.options() == before
        finally:
            G.close()
    finally:
        lb.lb_set_allocator(None, None)
