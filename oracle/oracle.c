/*
 * CPU oracle for frontier-driven BFS and SSSP with the load-balancing
 * schedules of Raval, Nasre, Kumar, R, Vadhiyar and Pingali, "Dynamic Load
 * Balancing Strategies for Graph Applications on GPUs" (arXiv 1711.00231).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow statement of what
 * the GPU path must produce.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does, and it shares no code, header, table or helper with the CUDA
 * library.
 *
 * What is computed, and where the paper defines it:
 *
 *  - BFS levels (Sec. II-B: BFS is the edge-distributive case "min level
 *    over level + 1"): level[v] = fewest directed edges on a path src -> v,
 *    -1 when v is unreachable.  Written as the textbook FIFO-queue BFS.
 *  - SSSP distances (Sec. II-B, Algorithm "SSSP Pseudocode illustrating
 *    Edge-Based Parallelism": dist starts at infinity, dist[src] = 0, and an
 *    edge lowers dist[dst] to dist[src] + weight).  The worklist relaxation
 *    converges to the unique least fixed point, i.e. the shortest-path
 *    distance, so the oracle is the plain definition computed by Dijkstra's
 *    algorithm (binary heap, lazy deletion, 64-bit sums).  Distances are
 *    reported in 32 bits: unreachable = 0xFFFFFFFF; a true distance
 *    >= 0xFFFFFFFE is reported as 0xFFFFFFFE and flags overflow.
 *  - Bellman-Ford and Floyd-Warshall: brute-force cross-checks for tiny
 *    graphs.
 *  - Invariant and parent-tree checkers for any claimed result.
 *  - Schedule artefacts of the strategies: the histogram MDT of Sec. III-B
 *    ("Automatic Determination of Node Splitting Threshold"), the per-thread
 *    (NodeOffset, EdgeOffset) start of workload decomposition (Sec. III-A,
 *    Algorithm "SSSP Pseudocode illustrating Workload Decomposition"), the
 *    node-splitting chunk sizes (Sec. III-B) and the hierarchical-processing
 *    sub-iteration schedule (Sec. III-C).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_UNREACHED 0xFFFFFFFFu
#define OR_SATURATED 0xFFFFFFFEu

/* ---------------------------------------------------------------- BFS --- */

/* FIFO BFS from src.  level[] receives hop counts, -1 for unreachable.
 * Returns the number of levels (eccentricity of src + 1), or -1 on a bad
 * argument or allocation failure. */
int64_t oracle_bfs(int64_t n, const int64_t *off, const int32_t *col, int32_t src, int32_t *level) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    int32_t maxlev = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                if (level[v] > maxlev) maxlev = level[v];
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return (int64_t)maxlev + 1;
}

/* ----------------------------------------------------------- Dijkstra --- */

typedef struct {
    uint64_t d;
    int32_t v;
} or_item;

typedef struct {
    or_item *a;
    int64_t len, cap;
} or_heap;

static int or_push(or_heap *h, uint64_t d, int32_t v) {
    if (h->len == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        or_item *na = (or_item *)realloc(h->a, (size_t)nc * sizeof(or_item));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    int64_t i = h->len++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].d <= d) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].d = d;
    h->a[i].v = v;
    return 0;
}

static or_item or_pop(or_heap *h) {
    or_item top = h->a[0];
    or_item last = h->a[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->len) break;
        if (c + 1 < h->len && h->a[c + 1].d < h->a[c].d) c++;
        if (h->a[c].d >= last.d) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->len > 0) h->a[i] = last;
    return top;
}

static int or_report(int64_t n, const uint64_t *d64, uint32_t *dist) {
    int overflow = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (d64[v] == UINT64_MAX) dist[v] = OR_UNREACHED;
        else if (d64[v] >= OR_SATURATED) { dist[v] = OR_SATURATED; overflow = 1; }
        else dist[v] = (uint32_t)d64[v];
    }
    return overflow;
}

/* Dijkstra from src with weights w (NULL = every weight 1).  Returns 0, 1
 * when some distance overflowed 32 bits (see the header), -1 on error. */
int oracle_dijkstra(int64_t n, const int64_t *off, const int32_t *col, const uint32_t *w, int32_t src,
                    uint32_t *dist) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!d) return -1;
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    or_heap h = {NULL, 0, 0};
    d[src] = 0;
    if (or_push(&h, 0, src)) { free(d); return -1; }
    while (h.len > 0) {
        or_item it = or_pop(&h);
        if (it.d != d[it.v]) continue; /* stale entry */
        int32_t u = it.v;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t v = col[e];
            uint64_t alt = d[u] + (w ? (uint64_t)w[e] : 1u);
            if (alt < d[v]) {
                d[v] = alt;
                if (or_push(&h, alt, v)) { free(h.a); free(d); return -1; }
            }
        }
    }
    free(h.a);
    int ov = or_report(n, d, dist);
    free(d);
    return ov;
}

/* ------------------------------------------------ brute-force checks --- */

/* Bellman-Ford: n-1 rounds over every edge, then one round that must change
 * nothing.  Returns 0/1 as oracle_dijkstra, -2 if the extra round changed a
 * distance (impossible for non-negative weights), -1 on error. */
int oracle_bellman_ford(int64_t n, const int64_t *off, const int32_t *col, const uint32_t *w, int32_t src,
                        uint32_t *dist) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!d) return -1;
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    d[src] = 0;
    int changed = 0;
    for (int64_t round = 0; round < n; ++round) {
        changed = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (d[u] == UINT64_MAX) continue;
            for (int64_t e = off[u]; e < off[u + 1]; ++e) {
                uint64_t alt = d[u] + (w ? (uint64_t)w[e] : 1u);
                if (alt < d[col[e]]) { d[col[e]] = alt; changed = 1; }
            }
        }
        if (round == n - 1 && changed) { free(d); return -2; }
        if (!changed) break;
    }
    int ov = or_report(n, d, dist);
    free(d);
    return ov;
}

/* Floyd-Warshall over all pairs (n <= 512); row src is returned.  Same
 * return convention as oracle_dijkstra. */
int oracle_floyd_warshall(int64_t n, const int64_t *off, const int32_t *col, const uint32_t *w, int32_t src,
                          uint32_t *dist) {
    if (n <= 0 || n > 512 || src < 0 || src >= n) return -1;
    uint64_t *D = (uint64_t *)malloc((size_t)(n * n) * sizeof(uint64_t));
    if (!D) return -1;
    for (int64_t i = 0; i < n * n; ++i) D[i] = UINT64_MAX;
    for (int64_t i = 0; i < n; ++i) D[i * n + i] = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t c = w ? (uint64_t)w[e] : 1u;
            if (c < D[u * n + col[e]]) D[u * n + col[e]] = c;
        }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) {
            if (D[i * n + k] == UINT64_MAX) continue;
            for (int64_t j = 0; j < n; ++j) {
                if (D[k * n + j] == UINT64_MAX) continue;
                uint64_t via = D[i * n + k] + D[k * n + j];
                if (via < D[i * n + j]) D[i * n + j] = via;
            }
        }
    int ov = or_report(n, D + (int64_t)src * n, dist);
    free(D);
    return ov;
}

/* ---------------------------------------------------------- checkers --- */

static inline uint64_t or_cap(uint64_t x) { return x >= OR_SATURATED ? OR_SATURATED : x; }

/* Checks a claimed distance vector (BFS levels pass as uint32 with w = NULL,
 * -1 reading as 0xFFFFFFFF):
 *   1: dist[src] != 0
 *   2: some edge u->v with u reached has dist[v] > min(dist[u]+w, 0xFFFFFFFE)
 *      (this includes a reached u with an unreached out-neighbour)
 *   3: some reached v != src has no in-edge achieving equality (not tight)
 * Returns 0 when all hold; *bad receives the offending vertex. */
int oracle_check_dist(int64_t n, const int64_t *off, const int32_t *col, const uint32_t *w, int32_t src,
                      const uint32_t *dist, int64_t *bad) {
    *bad = -1;
    if (n <= 0 || src < 0 || src >= n) return -1;
    if (dist[src] != 0) { *bad = src; return 1; }
    unsigned char *tight = (unsigned char *)calloc((size_t)n, 1);
    if (!tight) return -1;
    for (int64_t u = 0; u < n; ++u) {
        if (dist[u] == OR_UNREACHED) continue;
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            int32_t v = col[e];
            uint64_t alt = or_cap((uint64_t)dist[u] + (w ? (uint64_t)w[e] : 1u));
            if ((uint64_t)dist[v] > alt) { free(tight); *bad = v; return 2; }
            if ((uint64_t)dist[v] == alt) tight[v] = 1;
        }
    }
    for (int64_t v = 0; v < n; ++v)
        if (v != src && dist[v] != OR_UNREACHED && !tight[v]) { free(tight); *bad = v; return 3; }
    free(tight);
    return 0;
}

/* Checks a parent vector against a distance vector already known correct:
 *   1: parent[src] != src
 *   2: unreached v with parent[v] != -1
 *   3: reached v != src whose parent is out of range or unreached
 *   4: no edge parent[v] -> v with min(dist[p]+w, cap) == dist[v]
 *   5: following parents from v does not reach src (a cycle)
 * Returns 0 when all hold; *bad receives the offending vertex. */
int oracle_check_parents(int64_t n, const int64_t *off, const int32_t *col, const uint32_t *w, int32_t src,
                         const uint32_t *dist, const int32_t *parent, int64_t *bad) {
    *bad = -1;
    if (n <= 0 || src < 0 || src >= n) return -1;
    if (parent[src] != src) { *bad = src; return 1; }
    for (int64_t v = 0; v < n; ++v) {
        if (v == src) continue;
        if (dist[v] == OR_UNREACHED) {
            if (parent[v] != -1) { *bad = v; return 2; }
            continue;
        }
        int32_t p = parent[v];
        if (p < 0 || p >= n || dist[p] == OR_UNREACHED) { *bad = v; return 3; }
        int ok = 0;
        for (int64_t e = off[p]; e < off[p + 1] && !ok; ++e)
            if (col[e] == v && or_cap((uint64_t)dist[p] + (w ? (uint64_t)w[e] : 1u)) == dist[v]) ok = 1;
        if (!ok) { *bad = v; return 4; }
    }
    /* acyclicity: state 0 unknown, 1 on the current walk, 2 reaches src */
    unsigned char *st = (unsigned char *)calloc((size_t)n, 1);
    int32_t *path = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!st || !path) { free(st); free(path); return -1; }
    st[src] = 2;
    for (int64_t v = 0; v < n; ++v) {
        if (dist[v] == OR_UNREACHED || st[v] == 2) continue;
        int64_t len = 0;
        int32_t x = (int32_t)v;
        while (st[x] == 0) { st[x] = 1; path[len++] = x; x = parent[x]; }
        if (st[x] == 1) { free(st); free(path); *bad = v; return 5; }
        for (int64_t i = 0; i < len; ++i) st[path[i]] = 2;
    }
    free(st);
    free(path);
    return 0;
}

/* ------------------------------------------------- schedule artefacts --- */

/* Histogram MDT (Sec. III-B).  Degrees of the vertices with out-degree >= 1
 * fall into `bins` equal-width bins over (0, maxDeg]: bin k (1-based) holds
 * the degrees d with (k-1)*maxDeg < d*bins <= k*maxDeg.  binIndex is the
 * tallest bin (the smallest k on a tie) and
 * MDT = max(1, floor(binIndex * maxDeg / bins)).
 * Returns MDT (0 if no vertex has an out-edge), -1 on bad arguments. */
int64_t oracle_mdt(int64_t n, const int64_t *off, int32_t bins, int64_t *maxdeg_out, int32_t *bin_out,
                   int64_t *hist_out) {
    if (bins < 1 || n < 0) return -1;
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; ++u)
        if (off[u + 1] - off[u] > maxdeg) maxdeg = off[u + 1] - off[u];
    if (maxdeg_out) *maxdeg_out = maxdeg;
    if (maxdeg == 0) { if (bin_out) *bin_out = 0; return 0; }
    int64_t *hist = (int64_t *)calloc((size_t)bins + 1, sizeof(int64_t));
    if (!hist) return -1;
    for (int64_t u = 0; u < n; ++u) {
        int64_t d = off[u + 1] - off[u];
        if (d == 0) continue;
        /* smallest k with d*bins <= k*maxDeg */
        int64_t k = (d * (int64_t)bins + maxdeg - 1) / maxdeg;
        hist[k]++;
    }
    int32_t best = 1;
    for (int32_t k = 2; k <= bins; ++k)
        if (hist[k] > hist[best]) best = k;
    if (hist_out) memcpy(hist_out, hist + 1, (size_t)bins * sizeof(int64_t));
    free(hist);
    if (bin_out) *bin_out = best;
    int64_t mdt = ((int64_t)best * maxdeg) / bins;
    return mdt < 1 ? 1 : mdt;
}

/* Workload decomposition start offsets (Sec. III-A).  The F worklist nodes
 * have out-degrees deg[]; E = sum(deg) edges are cut into T contiguous blocks
 * of edgesPerThread = ceil(E / T).  Thread t (0-based) starts at global edge
 * t*edgesPerThread: node_off[t] is the worklist index whose edge range holds
 * it and edge_off[t] the position inside that node's edges; a thread whose
 * start is past the last edge gets (F, 0).  Returns edgesPerThread. */
int64_t oracle_wd_offsets(int64_t F, const int64_t *deg, int64_t T, int64_t *node_off, int64_t *edge_off) {
    if (T < 1 || F < 0) return -1;
    int64_t E = 0;
    for (int64_t i = 0; i < F; ++i) E += deg[i];
    int64_t ept = (E + T - 1) / T;
    for (int64_t t = 0; t < T; ++t) {
        int64_t s = t * ept;
        node_off[t] = F;
        edge_off[t] = 0;
        if (ept == 0 || s >= E) continue;
        int64_t before = 0;
        for (int64_t i = 0; i < F; ++i) {
            if (s < before + deg[i]) { node_off[t] = i; edge_off[t] = s - before; break; }
            before += deg[i];
        }
    }
    return ept;
}

/* Node splitting (Sec. III-B) of one node of out-degree deg at threshold
 * mdt: a node with deg > mdt becomes ceil(deg/mdt) nodes (the parent and its
 * children) owning consecutive runs of mdt edges, the last run the
 * remainder; otherwise it stays one node.  Writes the run lengths and
 * returns how many there are (at most cap are written). */
int64_t oracle_ns_chunks(int64_t deg, int64_t mdt, int64_t *sizes, int64_t cap) {
    if (mdt < 1 || deg < 0) return -1;
    if (deg <= mdt) {
        if (cap > 0) sizes[0] = deg;
        return 1;
    }
    int64_t k = (deg + mdt - 1) / mdt;
    for (int64_t i = 0; i < k && i < cap; ++i) sizes[i] = (i + 1 < k) ? mdt : deg - (k - 1) * mdt;
    return k;
}

/* Node counts after splitting a whole CSR at threshold mdt: returns the
 * number of child nodes created; *n_split receives how many nodes were
 * split (degree > mdt). */
int64_t oracle_ns_split(int64_t n, const int64_t *off, int64_t mdt, int64_t *n_split) {
    if (mdt < 1) return -1;
    int64_t children = 0, split = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t d = off[u + 1] - off[u];
        if (d > mdt) { split++; children += (d + mdt - 1) / mdt - 1; }
    }
    if (n_split) *n_split = split;
    return children;
}

/* Hierarchical processing of one super worklist (Sec. III-C).  The list
 * starts as the F nodes with out-degrees deg[].  Each step first checks the
 * list: if it holds fewer than `threshold` nodes, one workload-decomposition
 * step relaxes every edge the list's nodes have left and the iteration ends
 * (mode 1).  Otherwise a sub-iteration s (mode 0) lets every listed node
 * relax its next min(mdt, remaining) edges, i.e. edges s*mdt .. s*mdt+mdt-1
 * of its list; nodes with edges left form the next list.  The iteration ends
 * when the list is empty.  For each step k (at most cap) the function writes
 * the list size, the edges relaxed and the mode; it returns the step count.
 *
 * Hierarchy depth (Sec. III-C: a large sub-worklist "can be further
 * partitioned", the depth is tunable and the histogram MDT decides the
 * split).  Read here as: the lists of one super-iteration form a chain (the
 * super list, its sub-list, that list's sub-list, ...); each of the first
 * `depth` lists takes its own MDT -- the super list the given mdt (the
 * graph's histogram MDT), a sub-list the histogram rule applied to its
 * nodes' remaining degrees with `bins` bins -- and later lists keep the last
 * one.  depth = 1 is the single-MDT schedule of the HP algorithm. */
/* The histogram MDT rule of Sec. III-B over an array of degrees (the
 * remaining degrees of a sub-list): bins of equal width over (0, max], the
 * tallest bin k (1-based, smallest on a tie), MDT = max(1, floor(k max /
 * bins)); 0 when every degree is 0. */
static int64_t mdt_of_degrees(int64_t F, const int64_t *d, int32_t bins) {
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < F; ++i)
        if (d[i] > maxdeg) maxdeg = d[i];
    if (maxdeg == 0) return 0;
    int64_t *hist = (int64_t *)calloc((size_t)bins + 1, sizeof(int64_t));
    if (!hist) return -1;
    for (int64_t i = 0; i < F; ++i)
        if (d[i] > 0) hist[(d[i] * (int64_t)bins + maxdeg - 1) / maxdeg]++;
    int32_t best = 1;
    for (int32_t k = 2; k <= bins; ++k)
        if (hist[k] > hist[best]) best = k;
    free(hist);
    int64_t mdt = ((int64_t)best * maxdeg) / bins;
    return mdt < 1 ? 1 : mdt;
}

int64_t oracle_hp_schedule(int64_t F, const int64_t *deg, int64_t mdt, int64_t threshold, int32_t depth, int32_t bins,
                           int64_t *list_size, int64_t *edges, int32_t *mode, int64_t cap) {
    if (mdt < 1 || F < 0 || depth < 1 || bins < 1) return -1;
    int64_t *rem = (int64_t *)malloc((size_t)(F > 0 ? F : 1) * sizeof(int64_t));
    if (!rem) return -1;
    int64_t live = F;
    for (int64_t i = 0; i < F; ++i) rem[i] = deg[i];
    int64_t steps = 0;
    int64_t cur = mdt; /* edges per node in this sub-iteration */
    while (live > 0) {
        int64_t relaxed = 0;
        int32_t md;
        if (live < threshold) {
            for (int64_t i = 0; i < F; ++i) { relaxed += rem[i]; rem[i] = 0; }
            md = 1;
        } else {
            /* list number `steps` of the chain (0 = the super list, which
             * keeps the graph's MDT): within the first `depth` lists a
             * sub-list takes the MDT of its own remaining degrees */
            if (steps > 0 && steps < depth) {
                cur = mdt_of_degrees(F, rem, bins);
                if (cur < 1) { free(rem); return -1; }
            }
            for (int64_t i = 0; i < F; ++i) {
                int64_t take = rem[i] < cur ? rem[i] : cur;
                relaxed += take;
                rem[i] -= take;
            }
            md = 0;
        }
        if (steps < cap) {
            list_size[steps] = live;
            edges[steps] = relaxed;
            mode[steps] = md;
        }
        steps++;
        live = 0;
        for (int64_t i = 0; i < F; ++i) live += rem[i] > 0;
    }
    free(rem);
    return steps;
}
