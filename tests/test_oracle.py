"""Pins for the CPU oracle against things other than itself: brute force on
tiny graphs, a library routine (scipy.sparse.csgraph), closed forms on
paths / stars / complete graphs / grids, the worked examples and MDT values
the paper prints (tests/golden/), and planted mistakes that the invariant
checkers must catch."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def random_graph(rng, n, m, wmax=20, clean=True, zero_w=False):
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    w = rng.integers(0 if zero_w else 1, wmax + 1, m)
    return gg.from_edges(n, src, dst, w, clean=clean)


# ------------------------------------------------------------ brute force


@pytest.mark.parametrize("seed", range(40))
def test_bfs_dijkstra_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 48))
    m = int(rng.integers(0, 4 * n + 1))
    g = random_graph(rng, n, m, clean=bool(seed % 2), zero_w=(seed % 3 == 0))
    for src in {0, n - 1, int(rng.integers(0, n))}:
        lev, nlev = oracle.bfs(g, src)
        fw_unit, _ = oracle.floyd_warshall(g, src, unit=True)
        assert np.array_equal(lev.view(np.uint32), fw_unit)
        reached = lev >= 0
        assert nlev == lev[reached].max() + 1
        d, ov = oracle.dijkstra(g, src)
        bf, ov_bf = oracle.bellman_ford(g, src)
        fw, ov_fw = oracle.floyd_warshall(g, src)
        assert not ov and not ov_bf and not ov_fw
        assert np.array_equal(d, bf) and np.array_equal(d, fw)
        assert oracle.check_dist(g, src, d) == 0
        assert oracle.check_dist(g, src, lev, unit=True) == 0
        # unit-weight SSSP is BFS
        du, _ = oracle.dijkstra(g, src, unit=True)
        assert np.array_equal(du, lev.view(np.uint32))


@pytest.mark.parametrize("seed", range(6))
def test_against_scipy_csgraph(seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(100 + seed)
    n = 300
    g = random_graph(rng, n, 1500, wmax=1000, clean=True)
    A = sp.csr_matrix((g.weights.astype(np.float64), g.cols, g.offsets), shape=(n, n))
    for src in (0, 7, 299):
        ref = csgraph.dijkstra(A, directed=True, indices=src)
        d, _ = oracle.dijkstra(g, src)
        exp = np.where(np.isinf(ref), oracle.UNREACHED, ref).astype(np.uint64)
        assert np.array_equal(d.astype(np.uint64), exp)
        hops = csgraph.shortest_path(A, method="D", directed=True, unweighted=True, indices=src)
        lev, _ = oracle.bfs(g, src)
        assert np.array_equal(lev, np.where(np.isinf(hops), -1, hops).astype(np.int32))


def test_textbook_dijkstra_example():
    # The five-vertex weighted digraph used to illustrate Dijkstra's algorithm
    # in Cormen, Leiserson, Rivest and Stein, "Introduction to Algorithms"
    # (3rd ed., Sec. 24.3): s=0 t=1 x=2 y=3 z=4.
    e = [(0, 1, 10), (0, 3, 5), (1, 2, 1), (1, 3, 2), (2, 4, 4), (3, 1, 3), (3, 2, 9), (3, 4, 2), (4, 0, 7),
         (4, 2, 6)]
    g = gg.from_edges(5, [a for a, _, _ in e], [b for _, b, _ in e], [c for _, _, c in e])
    d, _ = oracle.dijkstra(g, 0)
    assert d.tolist() == [0, 8, 9, 5, 7]


# ------------------------------------------------------------ closed forms


def test_path_star_complete():
    n = 50
    path = gg.from_edges(n, np.arange(n - 1), np.arange(1, n), np.full(n - 1, 3))
    lev, nlev = oracle.bfs(path, 0)
    assert lev.tolist() == list(range(n)) and nlev == n
    d, _ = oracle.dijkstra(path, 0)
    assert d.tolist() == [3 * i for i in range(n)]
    lev, _ = oracle.bfs(path, 10)
    assert (lev[:10] == -1).all() and lev[10:].tolist() == list(range(n - 10))

    star = gg.from_edges(n, np.zeros(n - 1, int), np.arange(1, n), np.arange(1, n))
    lev, nlev = oracle.bfs(star, 0)
    assert lev[0] == 0 and (lev[1:] == 1).all() and nlev == 2
    d, _ = oracle.dijkstra(star, 0)
    assert d.tolist() == list(range(n))

    k = 12
    src = np.repeat(np.arange(k), k)
    dst = np.tile(np.arange(k), k)
    comp = gg.from_edges(k, src, dst, np.full(k * k, 5))
    assert comp.m == k * (k - 1)
    lev, _ = oracle.bfs(comp, 4)
    assert lev[4] == 0 and (np.delete(lev, 4) == 1).all()

    # complete binary tree: level of vertex i is floor(log2(i + 1))
    nb = 255
    tree = gg.from_edges(nb, np.arange(1, nb) // 2 - (np.arange(1, nb) % 2 == 0), np.arange(1, nb))
    lev, _ = oracle.bfs(tree, 0)
    assert lev.tolist() == [int(np.floor(np.log2(i + 1))) for i in range(nb)]


def test_grid_closed_form():
    R, C = 37, 53
    g = gg.grid(R, C, weights=None)
    assert g.m == 4 * R * C - 2 * R - 2 * C
    lev, nlev = oracle.bfs(g, 0)
    r, c = np.divmod(np.arange(R * C), C)
    assert np.array_equal(lev, (r + c).astype(np.int32))
    assert nlev == R + C - 1
    gw = gg.grid(R, C, weights=(7, 7))
    d, _ = oracle.dijkstra(gw, 0)
    assert np.array_equal(d, (7 * (r + c)).astype(np.uint32))
    # from the opposite corner
    d, _ = oracle.dijkstra(gw, R * C - 1)
    assert np.array_equal(d, (7 * ((R - 1 - r) + (C - 1 - c))).astype(np.uint32))


def test_overflow_saturates():
    big = 0x80000000
    g = gg.from_edges(4, [0, 1, 2], [1, 2, 3], [big, big - 3, 5])
    d, ov = oracle.dijkstra(g, 0)
    # 2^31, 2^32 - 3 (representable), then 2^32 + 2 saturates at 2^32 - 2
    assert d.tolist() == [0, big, 0xFFFFFFFD, oracle.SATURATED] and ov
    bf, ov2 = oracle.bellman_ford(g, 0)
    assert np.array_equal(bf, d) and ov2
    g2 = gg.from_edges(3, [0, 1], [1, 2], [big, big - 3])
    d2, ov3 = oracle.dijkstra(g2, 0)
    assert d2.tolist() == [0, big, 0xFFFFFFFD] and not ov3
    g3 = gg.from_edges(3, [0, 1], [1, 2], [big, big - 2])
    d3, ov4 = oracle.dijkstra(g3, 0)
    assert d3[2] == oracle.SATURATED and ov4


# ------------------------------------------------------ planted mistakes


def test_checkers_catch_planted_mistakes():
    rng = np.random.default_rng(7)
    g = random_graph(rng, 200, 1200, wmax=50)
    src = int(np.argmax(g.degrees()))
    d, _ = oracle.dijkstra(g, src)
    assert oracle.check_dist(g, src, d) == 0
    reached = np.flatnonzero((d != oracle.UNREACHED) & (np.arange(g.n) != src))
    v = int(reached[len(reached) // 2])
    bad = d.copy()
    bad[v] += 1                       # too large: some in-edge violates
    assert oracle.check_dist(g, src, bad)[0] == 2
    bad = d.copy()
    bad[v] -= 1                       # too small: not tight
    assert oracle.check_dist(g, src, bad)[0] in (2, 3)
    bad = d.copy()
    bad[src] = 1
    assert oracle.check_dist(g, src, bad)[0] == 1
    unreached = np.flatnonzero(d == oracle.UNREACHED)
    if unreached.size:
        bad = d.copy()
        bad[unreached[0]] = 5         # reached with no tight in-edge
        assert oracle.check_dist(g, src, bad)[0] in (2, 3)

    # a valid parent tree, then broken ones
    parent = np.full(g.n, -1, np.int32)
    parent[src] = src
    for u in range(g.n):
        if d[u] == oracle.UNREACHED:
            continue
        for e in range(g.offsets[u], g.offsets[u + 1]):
            x = g.cols[e]
            if x != src and parent[x] < 0 and int(d[u]) + int(g.weights[e]) == int(d[x]):
                parent[x] = u
    assert oracle.check_parents(g, src, d, parent) == 0
    p2 = parent.copy()
    p2[v] = src if parent[v] != src else int(reached[0])
    assert oracle.check_parents(g, src, d, p2) != 0 or parent[v] == p2[v]
    p3 = parent.copy()
    p3[src] = -1
    assert oracle.check_parents(g, src, d, p3)[0] == 1


def test_parent_cycle_detected_with_zero_weights():
    # 0 -> 1 (w 1), 1 <-> 2 with weight 0: dist 1 and 2 both 1; parents 1->2, 2->1 is a cycle
    g = gg.from_edges(3, [0, 1, 2], [1, 2, 1], [1, 0, 0])
    d, _ = oracle.dijkstra(g, 0)
    assert d.tolist() == [0, 1, 1]
    assert oracle.check_parents(g, 0, d, np.array([0, 0, 1], np.int32)) == 0
    assert oracle.check_parents(g, 0, d, np.array([0, 2, 1], np.int32))[0] == 5


# ------------------------------------------------- schedule artefacts


def test_wd_worked_example():
    gd = golden("wd_example.json")
    ept, node_off, edge_off = oracle.wd_offsets(gd["degrees"], gd["threads"])
    assert ept == gd["edges_per_thread"]
    # edge-to-thread assignment implied by the offsets: thread t takes global
    # edges [t*ept, (t+1)*ept)
    E = sum(gd["degrees"])
    starts = np.concatenate([[0], np.cumsum(gd["degrees"])])
    per_thread = []
    for t in range(gd["threads"]):
        cnt = [0] * len(gd["degrees"])
        for s in range(t * ept, min((t + 1) * ept, E)):
            cnt[int(np.searchsorted(starts, s, side="right") - 1)] += 1
        per_thread.append(cnt)
        # the offsets name the node/edge holding the thread's first edge
        i = int(node_off[t])
        assert starts[i] + edge_off[t] == t * ept
    t2 = gd["stated"]["thread"] - 1
    assert per_thread[t2] == [gd["stated"]["edges_from_first_node"], gd["stated"]["edges_from_second_node"]]
    assert all(sum(c) == ept for c in per_thread)
    assert (int(node_off[t2]), int(edge_off[t2])) == (0, 3)


def test_wd_offsets_edge_cases():
    ept, no, eo = oracle.wd_offsets([], 4)
    assert ept == 0 and no.tolist() == [0] * 4
    ept, no, eo = oracle.wd_offsets([0, 3, 0, 2], 2)
    assert ept == 3 and no.tolist() == [1, 3] and eo.tolist() == [0, 0]
    ept, no, eo = oracle.wd_offsets([1], 5)
    assert ept == 1 and no.tolist() == [0, 1, 1, 1, 1]


def test_hp_worked_example():
    gd = golden("hp_example.json")
    ls, ed, md = oracle.hp_schedule(gd["degrees"], gd["mdt"], threshold=0)
    exp = gd["derived_from_the_stated_rule"]
    assert len(ls) == exp["subiterations"]
    assert ed.tolist() == [sum(x) for x in exp["edges_per_node_per_subiteration"]]
    assert ls.tolist() == [2, 2, 1] and md.tolist() == [0, 0, 0]
    assert max(max(x) for x in exp["edges_per_node_per_subiteration"]) <= gd["max_edges_per_thread_per_subiteration"]
    # the paper's switch to workload decomposition below the block size (1024)
    ls, ed, md = oracle.hp_schedule(gd["degrees"], gd["mdt"], threshold=1024)
    assert md.tolist() == [1] and ed.tolist() == [12]
    # 100 edges left on one node at MDT 5 would take 20 sub-iterations
    # without the switch (the paper's own example of the occupancy problem)
    ls, ed, md = oracle.hp_schedule([100], 5, threshold=0)
    assert len(ls) == 20


def test_hp_depth_worked_examples():
    # hierarchy depth > 1: hand-worked cases of the rule (golden file), the
    # sub-list MDT re-derived with the pinned graph-MDT function on a CSR
    # whose degrees are the remaining degrees, and depth 1 = the plain schedule
    gd = golden("hp_depth_example.json")
    for case in gd["cases"]:
        ls, ed, md = oracle.hp_schedule(case["degrees"], case["mdt"], threshold=0, depth=case["depth"],
                                        bins=gd["bins"])
        assert ls.tolist() == case["list_sizes"] and ed.tolist() == case["edges"], case["name"]
        assert (md == 0).all() and ed.sum() == sum(case["degrees"])
        if "subiterations_at_depth_1" in case:
            assert len(oracle.hp_schedule(case["degrees"], case["mdt"], threshold=0)[0]) == \
                case["subiterations_at_depth_1"]
    rng = np.random.default_rng(11)
    for trial in range(30):
        deg = rng.integers(1, 400, int(rng.integers(1, 60)))
        deg[rng.random(deg.size) < 0.1] = rng.integers(1000, 5000)
        mdt0 = int(rng.integers(1, 50))
        plain = oracle.hp_schedule(deg, mdt0, threshold=0)
        d1 = oracle.hp_schedule(deg, mdt0, threshold=0, depth=1)
        assert all(np.array_equal(a, b) for a, b in zip(plain, d1))
        ls, ed, _ = oracle.hp_schedule(deg, mdt0, threshold=0, depth=2)
        assert ed.sum() == deg.sum()
        if len(ls) > 1:
            rem = np.maximum(deg - mdt0, 0)
            rem = rem[rem > 0]
            off = np.concatenate([[0], np.cumsum(rem)])
            mdt1 = oracle.mdt(off, 10)[0]
            assert ed[1] == np.minimum(rem, mdt1).sum(), trial


def test_ns_worked_example():
    gd = golden("ns_example.json")
    runs = oracle.ns_chunks(gd["degree"], gd["mdt"])
    assert len(runs) == gd["nodes_after_split"] and runs.tolist() == gd["runs"]
    assert oracle.ns_chunks(4, 4).tolist() == [4]
    assert oracle.ns_chunks(9, 4).tolist() == [4, 4, 1]
    assert oracle.ns_chunks(0, 4).tolist() == [0]
    off = np.concatenate([[0], np.cumsum([7, 3, 12, 0, 5])])
    assert oracle.ns_split(off, 4) == (1 + 2 + 1, 3)


def test_mdt_paper_values():
    gd = golden("mdt_paper_values.json")
    B = gd["bins"]
    rng = np.random.default_rng(3)
    for case in gd["cases"]:
        maxd = case["max_degree"]
        if case["graph"] == "rmat20":
            # heavy-tailed degrees: most nodes in the lowest tenth of the range
            deg = np.minimum(rng.zipf(1.8, 20000), maxd)
            deg = np.clip(deg, 1, maxd)
            deg[0] = maxd
        else:
            # ER-like: Poisson degrees with the mode at 3, capped at the max
            deg = np.clip(rng.poisson(3.4, 20000), 0, maxd)
            deg[0] = maxd
            assert np.bincount(deg)[1:].argmax() + 1 == 3
        off = np.concatenate([[0], np.cumsum(deg)])
        mdt, md, b, hist = oracle.mdt(off, B)
        assert md == maxd and b == case["tallest_bin_reading"] and mdt == case["mdt"]
        assert hist.sum() == (deg > 0).sum()


def test_mdt_rule_details():
    # equal-width bins over (0, maxDeg], bin k holds (k-1)*max < d*B <= k*max
    off = np.concatenate([[0], np.cumsum([10, 1, 1, 2, 0, 0, 0])])
    mdt, md, b, hist = oracle.mdt(off, 10)
    assert md == 10 and hist.tolist() == [2, 1, 0, 0, 0, 0, 0, 0, 0, 1] and b == 1 and mdt == 1
    # ties go to the smaller bin
    off = np.concatenate([[0], np.cumsum([20, 20, 2, 2])])
    mdt, md, b, hist = oracle.mdt(off, 10)
    assert b == 1 and mdt == 2
    # no edges at all
    assert oracle.mdt(np.zeros(5, np.int64), 10)[0] == 0
    # MDT never drops below 1
    off = np.concatenate([[0], np.cumsum([1] * 10 + [1000])])
    assert oracle.mdt(off, 10)[0] == 100
    off = np.concatenate([[0], np.cumsum([1, 1, 1, 3])])
    assert oracle.mdt(off, 10)[0] == 1


# ------------------------------------------------- generator sanity


def test_generators_are_clean_and_deterministic():
    g1 = gg.rmat(12, 8, seed=5)
    g2 = gg.rmat(12, 8, seed=5, nthreads=3)
    assert np.array_equal(g1.offsets, g2.offsets) and np.array_equal(g1.cols, g2.cols)
    assert np.array_equal(g1.weights, g2.weights)
    src = np.repeat(np.arange(g1.n), g1.degrees())
    assert (src != g1.cols).all()
    key = src.astype(np.int64) * g1.n + g1.cols
    assert (np.diff(key) > 0).all()     # sorted, no duplicates
    assert g1.weights.min() >= 1 and g1.weights.max() <= 255
    assert gg.draw(0, 0) == 0xE220A8397B1DCDAF  # first splitmix64 output for seed 0
    gr = gg.grid(5, 4)
    # undirected: weight(u,v) == weight(v,u)
    w = {}
    for u in range(gr.n):
        for e in range(gr.offsets[u], gr.offsets[u + 1]):
            w[(u, int(gr.cols[e]))] = int(gr.weights[e])
    assert all(w[(v, u)] == x for (u, v), x in w.items())
    s = gg.pick_sources(g1, 16, seed=1)
    assert len(set(s.tolist())) == 16 and (g1.degrees()[s] > 0).all()
    er = gg.erdos_renyi(1000, 4000, seed=2)
    assert er.m <= 4000 and er.m > 3900


def test_rmat_split_fraction_is_small():
    # Sec. III-B reports that fewer than 5% of the nodes undergo splitting at
    # the histogram MDT on its skewed graphs; the R-MAT stand-ins agree
    for scale in (14, 20):
        g = gg.rmat(scale, 16, seed=1)
        mdt = oracle.mdt(g.offsets, 10)[0]
        deg = np.diff(g.offsets)
        assert (deg > mdt).sum() / g.n < 0.05, scale
