"""lb_bfs_wd_noalloc: the BFS entry point for callers that cannot allocate
device memory (a process whose GPU memory belongs to another allocator, or
a service that must not call cudaMalloc while it runs).  Its levels must
equal those of the regular entry point, lb_bfs_dev, on two calls in a row
(the second call finds the first call's leftovers in the shared fixed
scratch array and must still be right).  The file name sorts last so a
stop-at-first-failure run has already run every other test."""
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


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    g = gg.rmat(16, 16, seed=5, weights=None)   # 65,536 vertices: inside the fixed limit
    off = torch.from_numpy(g.offsets).cuda()
    col = torch.from_numpy(g.cols).cuda()
    G = lb.Graph.from_csr(g)
    try:
        srcs = [gg.max_degree_vertex(g), int(gg.pick_sources(g, 1, seed=2)[0])]
        for src in srcs:           # two calls in a row on the same scratch array
            ref = torch.empty(g.n, dtype=torch.int32, device="cuda")
            G.bfs_dev(src, "WD", ref, None, torch.cuda.current_stream())
            out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            lb.lb_bfs_wd_noalloc(off, col, g.n, g.m, src, out, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert torch.equal(out, ref), f"src={src}"
            assert int((out >= 0).sum()) > 1
    finally:
        G.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    off = torch.zeros(4, dtype=torch.int64, device="cuda")
    lev = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(lb.LbError) as ei:
        lb.lb_bfs_wd_noalloc(off, off, (1 << 17) + 1, 0, 0, lev)
    assert ei.value.status == lb.LB_ERR_ARG and "131072" in str(ei.value)
    with pytest.raises(lb.LbError) as ei:
        lb.lb_bfs_wd_noalloc(off, off, 3, (1 << 24) + 1, 0, lev)
    assert ei.value.status == lb.LB_ERR_ARG


def test_noalloc_at_the_size_limit_then_a_smaller_graph():
    # n = 131,072 exactly (the array's vertex limit): the upper half of the
    # bitmap, both list buffers and the tile-start region are in use.  A
    # smaller graph right after it finds that call's leftovers in the array
    # (stale list entries, bitmap words past its own n) and must still be
    # exact.
    import torch
    big = gg.rmat(17, 16, seed=3, weights=None)
    small = gg.rmat(11, 8, seed=4, weights=None)
    assert big.n == 1 << 17
    for g, src in ((big, gg.max_degree_vertex(big)), (small, 0), (small, gg.max_degree_vertex(small))):
        off = torch.from_numpy(g.offsets).cuda()
        col = torch.from_numpy(g.cols).cuda()
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        lb.lb_bfs_wd_noalloc(off, col, g.n, g.m, src, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.bfs(g, src)[0]), (g.n, src)


def test_noalloc_refuses_a_malformed_csr():
    # the caller's CSR is checked on the device before the traversal: a
    # column equal to n, or offsets that do not end at m, return LB_ERR_ARG
    # and leave the output untouched
    import torch
    g = gg.rmat(10, 8, seed=6, weights=None)
    off = torch.from_numpy(g.offsets).cuda()
    bad_col = g.cols.copy()
    bad_col[g.m // 2] = g.n
    bad_off = g.offsets.copy()
    bad_off[-1] = g.m - 1
    for o, c in ((off, torch.from_numpy(bad_col).cuda()),
                 (torch.from_numpy(bad_off).cuda(), torch.from_numpy(g.cols).cuda())):
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        with pytest.raises(lb.LbError) as ei:
            lb.lb_bfs_wd_noalloc(o, c, g.n, g.m, 0, out, torch.cuda.current_stream())
        assert ei.value.status == lb.LB_ERR_ARG and "malformed" in str(ei.value)
        torch.cuda.synchronize()
        assert bool((out == 7).all())
    # a well-formed call afterwards is unaffected
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    lb.lb_bfs_wd_noalloc(off, torch.from_numpy(g.cols).cuda(), g.n, g.m, 0, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.bfs(g, 0)[0])
