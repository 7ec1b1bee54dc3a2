"""Small-list levels in one persistent launch (WD, option small_edges): while
the worklist has at most small_edges edges, levels run inside one
cooperative launch with a grid barrier between them.  Results must equal
the oracle's with the mode on, off, and with a threshold that makes the
lists move back and forth between the persistent launch and the per-level
launches; the trace must show which levels ran where.  The barrier's wait
is bounded: a CTA that never arrives (a test hook) makes the query return
LB_ERR_TIMEOUT and leaves the device usable."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from paper_1711_00231_gb300 import lb

pytestmark = pytest.mark.gpu

MODE_SMALL = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_00231_gb300 import _build
    _build.build()


def graphs():
    n = 3000
    path = gg.from_edges(n, np.arange(n - 1), np.arange(1, n), np.full(n - 1, 3))
    return [(gg.grid(300, 200, seed=2), [0, 30123]), (gg.rmat(14, 16, seed=1), [0, 17]), (path, [0, 1500]),
            (gg.rmat(18, 16, seed=4), None), (gg.erdos_renyi(50000, 200000, seed=3), [7])]


@pytest.mark.parametrize("loop_mode", [0, 1])
def test_small_list_levels_match_oracle(loop_mode):
    for g, srcs in graphs():
        if srcs is None:
            srcs = [gg.max_degree_vertex(g)]
        G = lb.Graph.from_csr(g)
        try:
            for se in (65536, 0, 300):
                G.set_options(small_edges=se, loop_mode=loop_mode)
                for src in srcs:
                    ref_lev, _ = oracle.bfs(g, src)
                    ref, _ = oracle.dijkstra(g, src)
                    lev = G.bfs(src, "WD")
                    assert np.array_equal(lev, ref_lev), (g.n, se, src)
                    st = G.stats()
                    assert st["status"] == 0
                    live = (ref_lev >= 0) & (g.degrees() > 0)
                    assert st["iterations"] == 1 + (int(ref_lev[live].max()) if live.any() else 0)
                    modes = G.trace()["mode"]
                    assert len(modes) == st["iterations"]
                    if se == 0:
                        assert not (modes == MODE_SMALL).any()
                    d, rc = G.sssp(src, "WD")
                    assert rc == lb.LB_OK and np.array_equal(d, ref), (g.n, se, src)
                # the high-diameter grid and the path run (almost) all levels in the persistent launch
                if se == 65536 and g.n in (60000, 3000):
                    G.bfs(srcs[0], "WD")
                    assert (G.trace()["mode"] == MODE_SMALL).mean() > 0.9
        finally:
            G.close()


def test_small_list_barrier_time_limit():
    g = gg.grid(64, 64, seed=1)
    ref_lev, _ = oracle.bfs(g, 0)
    G = lb.Graph.from_csr(g)
    try:
        G.set_options(test_barrier_skip=1)
        with pytest.raises(lb.LbError) as ei:
            G.bfs(0, "WD")
        assert ei.value.status == lb.LB_ERR_TIMEOUT
        G.set_options(test_barrier_skip=0)
        assert np.array_equal(G.bfs(0, "WD"), ref_lev)
        d, rc = G.sssp(0, "WD")
        assert rc == lb.LB_OK and np.array_equal(d, oracle.dijkstra(g, 0)[0])
    finally:
        G.close()
