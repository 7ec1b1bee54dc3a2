/*
 * Seeded synthetic graph inputs: R-MAT, Erdos-Renyi and 2-D grid graphs in
 * cleaned CSR form (self-loops and duplicate (u,v) pairs removed, each
 * adjacency list sorted by destination), plus integer edge weights and
 * source-vertex draws.
 *
 * This module holds none of the traversal arithmetic.  It is the one piece
 * of code that both the CPU oracle and the GPU path consume, so both see the
 * very same bytes.  All randomness comes from one counter-based generator:
 * the k-th output of splitmix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; constants as in Vigna's
 * public-domain splitmix64.c) seeded with a per-purpose stream seed.
 * Thresholds for the R-MAT quadrant draw are 64-bit integers, so the output
 * is bit-identical on x86-64 and AArch64 and independent of the thread count.
 *
 * The paper's own graphs (GTgraph R-MAT / ER, DIMACS road networks and the
 * Graph500 files of its Table II) are not available; these generators stand
 * in for them with the same shapes (skewed low-diameter R-MAT, random ER,
 * high-diameter near-uniform-degree grids standing in for road networks).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

typedef struct gg_csr {
    int64_t n;
    int64_t m;
    int64_t *offsets; /* n+1 */
    int32_t *cols;    /* m   */
    uint32_t *weights;/* m, or NULL */
} gg_csr;

/* splitmix64 output function (the finaliser applied to the Weyl state). */
static inline uint64_t gg_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* k-th (0-based) output of a splitmix64 generator whose state starts at s. */
uint64_t gg_draw(uint64_t s, uint64_t k) { return gg_mix64(s + (k + 1) * GG_GAMMA); }

/* Stream seed for a purpose tag: first output of splitmix64 seeded with
 * seed + tag*GAMMA.  Tags: 1 R-MAT quadrants, 2 edge weights, 3 sources,
 * 4 ER endpoints, 5 grid weights. */
uint64_t gg_stream(uint64_t seed, uint64_t tag) { return gg_draw(seed + tag * GG_GAMMA, 0); }

/* Uniform integer in [lo, hi] from a 64-bit draw (multiply-shift). */
static inline uint32_t gg_uniform(uint64_t x, uint32_t lo, uint32_t hi) {
    unsigned __int128 span = (unsigned __int128)((uint64_t)hi - lo + 1);
    return lo + (uint32_t)(((unsigned __int128)x * span) >> 64);
}

static int gg_threads(int req) {
    if (req > 0) return req;
    long p = sysconf(_SC_NPROCESSORS_ONLN);
    if (p < 1) p = 1;
    if (p > 64) p = 64;
    return (int)p;
}

/* ---------------- edge sources ---------------- */

typedef struct {
    int kind; /* 0 = R-MAT, 1 = ER */
    int scale;
    int64_t n;
    uint64_t t_a, t_ab, t_abc; /* cumulative 32-bit quadrant thresholds, r < t -> quadrant */
    uint64_t stream;
} gg_edgesrc;

static inline void gg_edge(const gg_edgesrc *es, int64_t i, uint32_t *pu, uint32_t *pv) {
    if (es->kind == 0) {
        /* one 64-bit draw serves two levels: the high 32 bits the even
         * level, the low 32 bits the odd one */
        uint32_t u = 0, v = 0;
        uint64_t per = (uint64_t)(es->scale + 1) / 2;
        uint64_t base = (uint64_t)i * per;
        uint32_t ta = (uint32_t)es->t_a, tab = (uint32_t)es->t_ab, tabc = (uint32_t)es->t_abc;
        uint64_t x = 0;
        for (int l = 0; l < es->scale; ++l) {
            if ((l & 1) == 0) x = gg_draw(es->stream, base + (uint64_t)(l >> 1));
            uint32_t r = (l & 1) ? (uint32_t)x : (uint32_t)(x >> 32);
            /* quadrant a: (0,0), b: (0,1), c: (1,0), d: (1,1); branch-free */
            uint32_t ga = r >= ta, gab = r >= tab, gabc = r >= tabc;
            u = (u << 1) | gab;
            v = (v << 1) | (ga ^ gab ^ gabc);
        }
        *pu = u;
        *pv = v;
    } else {
        uint64_t xu = gg_draw(es->stream, 2 * (uint64_t)i);
        uint64_t xv = gg_draw(es->stream, 2 * (uint64_t)i + 1);
        *pu = (uint32_t)(((unsigned __int128)xu * (uint64_t)es->n) >> 64);
        *pv = (uint32_t)(((unsigned __int128)xv * (uint64_t)es->n) >> 64);
    }
}

/* ---------------- parallel CSR build ---------------- */

typedef struct {
    const gg_edgesrc *es;
    int64_t e0, e1;       /* edge index range of this thread */
    uint32_t *cnt;        /* private per-vertex counter, later cursor */
    uint64_t *pairs;      /* generated (u << 32 | v), self-loops as all-ones */
    int32_t *raw;         /* scatter target */
    const int64_t *roff;  /* raw offsets */
    int phase;
} gg_work;

#define GG_NOEDGE 0xFFFFFFFFFFFFFFFFULL

static void *gg_count_or_scatter(void *arg) {
    gg_work *w = (gg_work *)arg;
    if (w->phase == 0) {
        for (int64_t i = w->e0; i < w->e1; ++i) {
            uint32_t u, v;
            gg_edge(w->es, i, &u, &v);
            if (u == v) { w->pairs[i] = GG_NOEDGE; continue; }
            w->pairs[i] = ((uint64_t)u << 32) | v;
            w->cnt[u]++;
        }
    } else {
        for (int64_t i = w->e0; i < w->e1; ++i) {
            uint64_t p = w->pairs[i];
            if (p == GG_NOEDGE) continue;
            uint32_t u = (uint32_t)(p >> 32);
            int64_t pos = w->roff[u] + (int64_t)(w->cnt[u]++);
            w->raw[pos] = (int32_t)(uint32_t)p;
        }
    }
    return NULL;
}

static void gg_insertion(uint32_t *a, int64_t len) {
    for (int64_t i = 1; i < len; ++i) {
        uint32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

/* LSD radix sort on 8-bit digits; passes above the key range are skipped. */
static void gg_radix(uint32_t *a, uint32_t *tmp, int64_t len, uint32_t maxkey) {
    int passes = 1;
    while (passes < 4 && (maxkey >> (8 * passes)) != 0) passes++;
    uint32_t *src = a, *dst = tmp;
    for (int p = 0; p < passes; ++p) {
        int64_t count[257];
        memset(count, 0, sizeof(count));
        int sh = 8 * p;
        for (int64_t i = 0; i < len; ++i) count[((src[i] >> sh) & 255u) + 1]++;
        for (int d = 0; d < 256; ++d) count[d + 1] += count[d];
        for (int64_t i = 0; i < len; ++i) dst[count[(src[i] >> sh) & 255u]++] = src[i];
        uint32_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)len * sizeof(uint32_t));
}

typedef struct {
    int64_t n;
    const int64_t *roff;
    int32_t *raw;
    int64_t *newdeg;
    int64_t *next_row; /* shared dynamic row counter */
    int64_t maxdeg;
} gg_sortwork;

#define GG_ROW_CHUNK 2048

static void *gg_sort_rows(void *arg) {
    gg_sortwork *w = (gg_sortwork *)arg;
    uint32_t *tmp = (uint32_t *)malloc((size_t)(w->maxdeg > 0 ? w->maxdeg : 1) * sizeof(uint32_t));
    if (!tmp) return (void *)1;
    for (;;) {
        int64_t r0 = __atomic_fetch_add(w->next_row, GG_ROW_CHUNK, __ATOMIC_RELAXED);
        if (r0 >= w->n) break;
        int64_t r1 = r0 + GG_ROW_CHUNK < w->n ? r0 + GG_ROW_CHUNK : w->n;
        for (int64_t u = r0; u < r1; ++u) {
            uint32_t *row = (uint32_t *)(w->raw + w->roff[u]);
            int64_t len = w->roff[u + 1] - w->roff[u];
            if (len <= 1) { w->newdeg[u] = len; continue; }
            if (len <= 48) {
                gg_insertion(row, len);
            } else {
                uint32_t mx = 0;
                for (int64_t i = 0; i < len; ++i) if (row[i] > mx) mx = row[i];
                gg_radix(row, tmp, len, mx);
            }
            int64_t k = 1;
            for (int64_t i = 1; i < len; ++i)
                if (row[i] != row[k - 1]) row[k++] = row[i];
            w->newdeg[u] = k;
        }
    }
    free(tmp);
    return NULL;
}

typedef struct {
    int64_t u0, u1;
    const int64_t *roff, *noff;
    const int32_t *raw;
    int32_t *cols;
} gg_compactwork;

static void *gg_compact(void *arg) {
    gg_compactwork *w = (gg_compactwork *)arg;
    for (int64_t u = w->u0; u < w->u1; ++u) {
        int64_t len = w->noff[u + 1] - w->noff[u];
        memcpy(w->cols + w->noff[u], w->raw + w->roff[u], (size_t)len * sizeof(int32_t));
    }
    return NULL;
}

typedef struct {
    int64_t e0, e1;
    uint64_t stream;
    uint32_t lo, hi;
    uint32_t *w;
} gg_weightwork;

static void *gg_weights(void *arg) {
    gg_weightwork *w = (gg_weightwork *)arg;
    for (int64_t e = w->e0; e < w->e1; ++e) w->w[e] = gg_uniform(gg_draw(w->stream, (uint64_t)e), w->lo, w->hi);
    return NULL;
}

void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->offsets);
    free(g->cols);
    free(g->weights);
    g->offsets = NULL;
    g->cols = NULL;
    g->weights = NULL;
}

/* Returns 0 on success, -1 on allocation failure, -2 on bad arguments. */
static int gg_build(const gg_edgesrc *es, int64_t n, int64_t nedges, uint64_t seed, int weighted,
                    uint32_t wlo, uint32_t whi, int nthreads, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (n <= 0 || n > (int64_t)INT32_MAX || nedges < 0 || (weighted && wlo > whi)) return -2;
    int T = gg_threads(nthreads);
    if ((int64_t)T > nedges / 4096 + 1) T = (int)(nedges / 4096 + 1);
    pthread_t th[64];
    gg_work wk[64];
    uint32_t **cnt = (uint32_t **)calloc((size_t)T, sizeof(uint32_t *));
    int64_t *roff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!cnt || !roff) { free(cnt); free(roff); return -1; }
    int rc = 0;
    for (int t = 0; t < T; ++t) {
        cnt[t] = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
        if (!cnt[t]) rc = -1;
    }
    int32_t *raw = NULL;
    int64_t *newdeg = NULL;
    int64_t *noff = NULL;
    uint64_t *pairs = (uint64_t *)malloc((size_t)(nedges > 0 ? nedges : 1) * sizeof(uint64_t));
    if (!pairs) rc = -1;
    if (rc) goto fail;
    for (int t = 0; t < T; ++t) {
        wk[t].es = es;
        wk[t].e0 = nedges * t / T;
        wk[t].e1 = nedges * (t + 1) / T;
        wk[t].cnt = cnt[t];
        wk[t].pairs = pairs;
        wk[t].phase = 0;
        pthread_create(&th[t], NULL, gg_count_or_scatter, &wk[t]);
    }
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    /* raw offsets, and per-thread cursors turned into exclusive starts */
    roff[0] = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t s = 0;
        for (int t = 0; t < T; ++t) {
            uint32_t c = cnt[t][u];
            cnt[t][u] = (uint32_t)s;
            s += c;
        }
        roff[u + 1] = roff[u] + s;
    }
    int64_t mraw = roff[n];
    raw = (int32_t *)malloc((size_t)(mraw > 0 ? mraw : 1) * sizeof(int32_t));
    if (!raw) { rc = -1; goto fail; }
    for (int t = 0; t < T; ++t) {
        wk[t].phase = 1;
        wk[t].raw = raw;
        wk[t].roff = roff;
        pthread_create(&th[t], NULL, gg_count_or_scatter, &wk[t]);
    }
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < T; ++t) { free(cnt[t]); cnt[t] = NULL; }
    free(pairs);
    pairs = NULL;
    newdeg = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!newdeg) { rc = -1; goto fail; }
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t d = roff[u + 1] - roff[u];
        if (d > maxdeg) maxdeg = d;
    }
    {
        int64_t next_row = 0;
        gg_sortwork sw = {n, roff, raw, newdeg, &next_row, maxdeg};
        int Ts = gg_threads(nthreads);
        for (int t = 0; t < Ts; ++t) pthread_create(&th[t], NULL, gg_sort_rows, &sw);
        for (int t = 0; t < Ts; ++t) {
            void *r = NULL;
            pthread_join(th[t], &r);
            if (r) rc = -1;
        }
        if (rc) goto fail;
    }
    noff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!noff) { rc = -1; goto fail; }
    noff[0] = 0;
    for (int64_t u = 0; u < n; ++u) noff[u + 1] = noff[u] + newdeg[u];
    free(newdeg);
    newdeg = NULL;
    int64_t m = noff[n];
    out->cols = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!out->cols) { rc = -1; goto fail; }
    {
        int Ts = gg_threads(nthreads);
        gg_compactwork cw[64];
        for (int t = 0; t < Ts; ++t) {
            cw[t].u0 = n * t / Ts;
            cw[t].u1 = n * (t + 1) / Ts;
            cw[t].roff = roff;
            cw[t].noff = noff;
            cw[t].raw = raw;
            cw[t].cols = out->cols;
            pthread_create(&th[t], NULL, gg_compact, &cw[t]);
        }
        for (int t = 0; t < Ts; ++t) pthread_join(th[t], NULL);
    }
    free(raw);
    raw = NULL;
    free(roff);
    roff = NULL;
    out->n = n;
    out->m = m;
    out->offsets = noff;
    noff = NULL;
    if (weighted) {
        out->weights = (uint32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
        if (!out->weights) { rc = -1; goto fail; }
        int Ts = gg_threads(nthreads);
        gg_weightwork ww[64];
        uint64_t ws = gg_stream(seed, 2);
        for (int t = 0; t < Ts; ++t) {
            ww[t].e0 = m * t / Ts;
            ww[t].e1 = m * (t + 1) / Ts;
            ww[t].stream = ws;
            ww[t].lo = wlo;
            ww[t].hi = whi;
            ww[t].w = out->weights;
            pthread_create(&th[t], NULL, gg_weights, &ww[t]);
        }
        for (int t = 0; t < Ts; ++t) pthread_join(th[t], NULL);
    }
    free(cnt);
    return 0;
fail:
    if (cnt) for (int t = 0; t < T; ++t) free(cnt[t]);
    free(pairs);
    free(cnt);
    free(roff);
    free(raw);
    free(newdeg);
    free(noff);
    gg_free(out);
    return rc;
}

/* R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): nedges generated edges
 * over 2^scale vertices; at each of the scale levels one draw picks the
 * quadrant (a: top-left, b: top-right, c: bottom-left, d: bottom-right) and
 * appends one bit to the source (row) and destination (column) ids, most
 * significant bit first.  Edge i uses draws i*ceil(scale/2) + j; the high 32
 * bits of draw j decide level 2j and the low 32 bits level 2j+1.  t_a, t_ab,
 * t_abc are floor(a*2^32), floor((a+b)*2^32), floor((a+b+c)*2^32).  No vertex
 * permutation, no noise. */
int gg_rmat(int scale, int64_t nedges, uint64_t t_a, uint64_t t_ab, uint64_t t_abc, uint64_t seed,
            int weighted, uint32_t wlo, uint32_t whi, int nthreads, gg_csr *out) {
    if (scale < 1 || scale > 30) return -2;
    gg_edgesrc es;
    memset(&es, 0, sizeof(es));
    es.kind = 0;
    es.scale = scale;
    es.n = (int64_t)1 << scale;
    es.t_a = t_a;
    es.t_ab = t_ab;
    es.t_abc = t_abc;
    es.stream = gg_stream(seed, 1);
    return gg_build(&es, es.n, nedges, seed, weighted, wlo, whi, nthreads, out);
}

/* Erdos-Renyi G(n, M)-style: nedges independent uniform (u, v) draws, then
 * self-loops and duplicates removed. */
int gg_er(int64_t n, int64_t nedges, uint64_t seed, int weighted, uint32_t wlo, uint32_t whi, int nthreads,
          gg_csr *out) {
    gg_edgesrc es;
    memset(&es, 0, sizeof(es));
    es.kind = 1;
    es.n = n;
    es.stream = gg_stream(seed, 4);
    return gg_build(&es, n, nedges, seed, weighted, wlo, whi, nthreads, out);
}

/* rows x cols 4-neighbour grid, vertex id r*cols + c, both directions of
 * every undirected edge present, neighbours in increasing id order.  The
 * weight of the undirected edge {(r,c),(r,c+1)} is drawn at counter
 * 2*(r*cols+c), that of {(r,c),(r+1,c)} at 2*(r*cols+c)+1, and both
 * directions carry the same weight. */
int gg_grid(int64_t rows, int64_t cols, uint64_t seed, int weighted, uint32_t wlo, uint32_t whi, gg_csr *out) {
    memset(out, 0, sizeof(*out));
    if (rows <= 0 || cols <= 0 || rows * cols > (int64_t)INT32_MAX || (weighted && wlo > whi)) return -2;
    int64_t n = rows * cols;
    out->offsets = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!out->offsets) return -1;
    out->offsets[0] = 0;
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            int64_t id = r * cols + c;
            int d = (r > 0) + (c > 0) + (c + 1 < cols) + (r + 1 < rows);
            out->offsets[id + 1] = out->offsets[id] + d;
        }
    int64_t m = out->offsets[n];
    out->cols = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (weighted) out->weights = (uint32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    if (!out->cols || (weighted && !out->weights)) { gg_free(out); return -1; }
    uint64_t ws = gg_stream(seed, 5);
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            int64_t id = r * cols + c;
            int64_t e = out->offsets[id];
            /* (neighbour id, undirected key) in increasing neighbour id */
            if (r > 0) {
                out->cols[e] = (int32_t)(id - cols);
                if (weighted) out->weights[e] = gg_uniform(gg_draw(ws, 2 * (uint64_t)(id - cols) + 1), wlo, whi);
                ++e;
            }
            if (c > 0) {
                out->cols[e] = (int32_t)(id - 1);
                if (weighted) out->weights[e] = gg_uniform(gg_draw(ws, 2 * (uint64_t)(id - 1)), wlo, whi);
                ++e;
            }
            if (c + 1 < cols) {
                out->cols[e] = (int32_t)(id + 1);
                if (weighted) out->weights[e] = gg_uniform(gg_draw(ws, 2 * (uint64_t)id), wlo, whi);
                ++e;
            }
            if (r + 1 < rows) {
                out->cols[e] = (int32_t)(id + cols);
                if (weighted) out->weights[e] = gg_uniform(gg_draw(ws, 2 * (uint64_t)id + 1), wlo, whi);
                ++e;
            }
        }
    out->n = n;
    out->m = m;
    return 0;
}

/* Uniform weights U[lo,hi] for an existing CSR of m edges (counter = edge
 * index, stream tag 2), for graphs built outside this module. */
void gg_fill_weights(int64_t m, uint64_t seed, uint32_t wlo, uint32_t whi, uint32_t *w) {
    uint64_t ws = gg_stream(seed, 2);
    for (int64_t e = 0; e < m; ++e) w[e] = gg_uniform(gg_draw(ws, (uint64_t)e), wlo, whi);
}

/* Up to `count` distinct sources drawn uniformly among the vertices with
 * out-degree > 0 (stream tag 3, draws k = 0, 1, 2, ...; a repeat is redrawn).
 * Returns the number written. */
int64_t gg_pick_sources(int64_t n, const int64_t *offsets, int64_t count, uint64_t seed, int32_t *out) {
    int64_t nz = 0;
    for (int64_t u = 0; u < n; ++u) nz += offsets[u + 1] > offsets[u];
    if (nz == 0 || count <= 0) return 0;
    int32_t *cand = (int32_t *)malloc((size_t)nz * sizeof(int32_t));
    if (!cand) return -1;
    int64_t k = 0;
    for (int64_t u = 0; u < n; ++u)
        if (offsets[u + 1] > offsets[u]) cand[k++] = (int32_t)u;
    if (count > nz) count = nz;
    uint64_t ss = gg_stream(seed, 3);
    int64_t got = 0;
    for (uint64_t draw = 0; got < count; ++draw) {
        uint64_t x = gg_draw(ss, draw);
        int32_t v = cand[(int64_t)(((unsigned __int128)x * (uint64_t)nz) >> 64)];
        int dup = 0;
        for (int64_t j = 0; j < got; ++j)
            if (out[j] == v) { dup = 1; break; }
        if (!dup) out[got++] = v;
    }
    free(cand);
    return got;
}
