"""Failure handling without a GPU fault: device allocations refused through
the allocator hook (at graph creation and at each strategy's first
workspace), and a serving engine that cannot fit one query slot.  Every
failure must come back as LB_ERR_OOM, leave nothing allocated, and a later
attempt with memory available must give exact results."""
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


class Hook:
    """Device allocator backed by torch tensors that can be told to refuse."""

    def __init__(self):
        self.keep = {}
        self.refuse = False
        self.refused = 0

    def alloc(self, size):
        import torch
        if self.refuse:
            self.refused += 1
            return 0
        t = torch.empty(max(size, 1), dtype=torch.uint8, device="cuda")
        self.keep[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr):
        self.keep.pop(ptr, None)


def test_refused_allocations_are_reported_and_recoverable():
    g = gg.rmat(12, 8, seed=2)
    ref_lev = oracle.bfs(g, 0)[0]
    ref_d = oracle.dijkstra(g, 0)[0]
    h = Hook()
    lb.lb_set_allocator(h.alloc, h.free)
    try:
        h.refuse = True
        with pytest.raises(lb.LbError) as ei:
            lb.Graph.from_csr(g)
        assert ei.value.status == lb.LB_ERR_OOM and h.refused >= 1
        assert not h.keep
        h.refuse = False
        G = lb.Graph.from_csr(g)
        try:
            for s in ["WD", "EP", "NS_PHYS", "HP", "BS"]:
                G.release()                      # every strategy starts from an empty workspace
                h.refuse = True
                with pytest.raises(lb.LbError) as ei:
                    G.bfs(0, s)
                assert ei.value.status == lb.LB_ERR_OOM, s
                h.refuse = False
                assert np.array_equal(G.bfs(0, s), ref_lev), s
                d, rc = G.sssp(0, s)
                assert rc == lb.LB_OK and np.array_equal(d, ref_d), s
        finally:
            G.close()
        assert not h.keep                        # everything allocated through the hook came back
    finally:
        lb.lb_set_allocator(None, None)


def test_allocation_refused_part_way_through_a_workspace():
    # refuse the k-th allocation of a first query for every k until one
    # succeeds: whatever was allocated before the refusal must be released
    # or reused, and the query must then be exact
    g = gg.rmat(11, 8, seed=4)
    ref_lev = oracle.bfs(g, 3)[0]
    for s in ["WD", "EP", "HP"]:
        k = 0
        while True:
            state = {"armed": False, "n": 0}
            h = Hook()

            def alloc(size, h=h, state=state, k=k):
                if state["armed"]:
                    state["n"] += 1
                    h.refuse = state["n"] == k + 1     # refuse the query's (k+1)-th allocation only
                return h.alloc(size)
            lb.lb_set_allocator(alloc, h.free)
            try:
                G = lb.Graph.from_csr(g)
                state["armed"] = True
                try:
                    try:
                        lev = G.bfs(3, s)
                        ok = True
                    except lb.LbError as e:
                        assert e.status == lb.LB_ERR_OOM
                        ok = False
                        lev = G.bfs(3, s)        # the retry completes the workspace
                    assert np.array_equal(lev, ref_lev), (s, k)
                finally:
                    G.close()
                assert not h.keep, (s, k)
            finally:
                lb.lb_set_allocator(None, None)
            if ok:
                break
            k += 1
            assert k < 40


def test_server_admission_by_free_memory_refuses_when_nothing_fits():
    g = gg.rmat(12, 8, seed=2)
    G = lb.Graph.from_csr(g)
    try:
        with pytest.raises(lb.LbError) as ei:
            sv.Server([G], mem_fraction=1e-9)
        assert ei.value.status == lb.LB_ERR_OOM
        S = sv.Server([G], slots=4096, mem_fraction=0.001)   # a pool of 0.1% of free HBM
        try:
            info = S.info()
            assert info["slots"] == 4096
            assert info["slot_bytes"] <= info["pool_bytes"] <= 0.001 * 300e9
            assert info["pool_bytes"] < 4096 * info["slot_bytes"]   # memory, not the slot count, bounds admission
            assert info["pool_free"] == info["pool_bytes"] and info["pending"] == 0
        finally:
            S.close()
    finally:
        G.close()
