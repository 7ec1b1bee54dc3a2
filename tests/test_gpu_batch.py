"""Batched host-output queries (lb_bfs_batch / lb_sssp_batch): k results
written row by row to host memory while the next query runs.  Every row
must equal the oracle's levels / distances for its source, for pinned and
pageable output, odd and even k (the two device result buffers alternate),
and the call must leave the output alone when a source is invalid."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1711_00231_gb300 import lb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_00231_gb300 import _build
    _build.build()


def pinned(shape, dtype):
    import torch
    t = torch.empty(int(np.prod(shape)), dtype=torch.int32, pin_memory=True)
    return t.numpy().view(dtype).reshape(shape), t


@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("strategy", ["WD", "BS", "EP", "HP"])
def test_batch_rows_match_oracle(k, strategy):
    g = gg.rmat(14, 16, seed=1)
    srcs = [int(s) for s in gg.pick_sources(g, k, seed=3)]
    G = lb.Graph.from_csr(g)
    try:
        lev, keep = pinned((k, g.n), np.int32)
        G.bfs_batch(srcs, strategy, lev)
        dist, rc = G.sssp_batch(srcs, strategy)   # pageable output
        assert rc == lb.LB_OK
        for i, s in enumerate(srcs):
            assert np.array_equal(lev[i], oracle.bfs(g, s)[0]), (strategy, i, s)
            assert np.array_equal(dist[i], oracle.dijkstra(g, s)[0]), (strategy, i, s)
        assert G.stats()["status"] == 0
    finally:
        G.close()


def test_batch_equals_single_queries_on_rmat20():
    # larger results (4 MiB each): the copy of row i overlaps query i + 1
    g = gg.rmat(20, 16, seed=1)
    srcs = [int(s) for s in gg.pick_sources(g, 7, seed=1)]
    G = lb.Graph.from_csr(g)
    try:
        dist, keep = pinned((len(srcs), g.n), np.uint32)
        _, rc = G.sssp_batch(srcs, "WD", dist)
        assert rc == lb.LB_OK
        lev = G.bfs_batch(srcs, "WD")
        for i, s in enumerate(srcs):
            assert np.array_equal(dist[i], G.sssp(s, "WD")[0]), i
            assert np.array_equal(lev[i], G.bfs(s, "WD")), i
        for i in (0, len(srcs) - 1):
            assert np.array_equal(dist[i], oracle.dijkstra(g, srcs[i])[0]), i
    finally:
        G.close()


def test_batch_reports_overflow_and_bad_sources():
    big = 0x80000000
    g = gg.from_edges(5, [0, 1, 2, 0], [1, 2, 3, 4], [big, big - 3, 5, 1])
    G = lb.Graph.from_csr(g)
    try:
        # source 2 cannot overflow, source 0 does: the first failing query
        # sets the status, every row is still written
        out, rc = G.sssp_batch([2, 0, 2])
        assert rc == lb.LB_ERR_OVERFLOW
        assert "query 1" in lb.lib().lb_last_error().decode()
        for i, s in enumerate([2, 0, 2]):
            assert np.array_equal(out[i], oracle.dijkstra(g, s)[0])
        sentinel = np.full((3, g.n), 7, dtype=np.int32)
        with pytest.raises(lb.LbError) as ei:
            G.bfs_batch([0, g.n, 1], "WD", sentinel)
        assert ei.value.status == lb.LB_ERR_ARG and "query 1" in str(ei.value)
        assert bool((sentinel == 7).all())
        assert G.bfs_batch([], "WD").shape == (0, g.n)
    finally:
        G.close()
