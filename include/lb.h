/*
 * lb.h -- C ABI of the GB300 (sm_103a) frontier BFS / SSSP library with the
 * dynamic load-balancing strategies of "Dynamic Load Balancing Strategies
 * for Graph Applications on GPUs" (Raval, Nasre, Kumar, R, Vadhiyar,
 * Pingali; arXiv 1711.00231).
 *
 * The problem statement follows the paper's Algorithms "SSSP Pseudocode
 * illustrating Edge-Based Parallelism" and "... Workload Decomposition":
 * a directed graph in CSR form (Sec. I and II-B: N + E elements, N + 2E with
 * weights), dist[] initialised to infinity, dist[source] = 0, and worklist
 * iterations that relax the out-edges of the active nodes until the worklist
 * is empty.  BFS is the unit-weight case (Sec. II-B: min level distributes
 * over level + 1).
 *
 * Conventions for every entry point:
 *  - Status codes only; no exception or signal ever crosses the ABI.  On an
 *    error, lb_last_error() returns a message for the calling thread.
 *  - Host pointers are plain host memory; "_dev" pointers are device
 *    pointers on the graph's device; "stream" is a cudaStream_t (NULL = the
 *    legacy default stream).
 *  - All integer arithmetic is exact: levels and distances are identical to
 *    the plain definitions (fewest hops; least sum of weights) for every
 *    strategy and every schedule.
 *  - Calls on one lb_graph are serialised by the library (a per-graph lock
 *    plus a stream-ordering event); different graphs may be used
 *    concurrently from different threads.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_graph lb_graph; /* opaque; owns device copies of the CSR */

/* Work distribution strategies.  Baselines (Sec. II) and the paper's three
 * dynamic strategies (Sec. III). */
typedef enum lb_strategy {
    LB_BS = 0,  /* node-based: one thread per worklist node, all its edges
                   (Sec. II-A; the LonestarGPU-style baseline "BS") */
    LB_EP = 1,  /* edge-based: one thread per worklist edge of a COO graph;
                   an updated node's edges are pushed with one reservation
                   (work chunking, Sec. II-B and IV-D) */
    LB_WD = 2,  /* workload decomposition: the worklist's edges are cut into
                   equal contiguous blocks found from the prefix sum of
                   worklist out-degrees (Sec. III-A) */
    LB_NS = 3,  /* node splitting: a node of out-degree d > MDT is served as
                   ceil(d/MDT) nodes of at most MDT edges; MDT from the
                   degree histogram (Sec. III-B) */
    LB_HP = 4,  /* hierarchical processing: sub-iterations that relax at most
                   MDT edges per node, switching to WD below a list-size
                   threshold (Sec. III-C) */
    LB_NS_PHYS = 5, /* node splitting with physical child nodes: ids n..n+S-1,
                   child lists, distances mirrored from the parent with
                   extra atomics, as in the paper's NS algorithm; same
                   results as LB_NS, more memory and atomics */
    LB_EP_NOCHUNK = 6, /* EP without work chunking: one atomic reservation per
                   pushed edge, the default the paper's Sec. IV-D compares
                   work chunking against */
    LB_AUTO = 15 /* the library's choice (currently LB_WD) */
} lb_strategy;

typedef enum lb_status {
    LB_OK = 0,
    LB_ERR_ARG = -1,         /* invalid argument or malformed CSR */
    LB_ERR_OOM = -2,         /* device allocation failed */
    LB_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    LB_ERR_OVERFLOW = -4,    /* some shortest distance is >= 2^32 - 2 */
    LB_ERR_TIMEOUT = -5,     /* iteration cap reached (never expected) */
    LB_ERR_UNSUPPORTED = -6, /* e.g. lb_sssp on a graph created without weights */
    LB_ERR_INTERNAL = -7     /* a device-side consistency check failed */
} lb_status;

typedef enum lb_kind { LB_KIND_BFS = 0, LB_KIND_SSSP = 1 } lb_kind;

/* Tunables.  Zero fields take the defaults shown. */
typedef struct lb_options {
    int32_t hist_bins;     /* HistogramBinCount of the MDT heuristic (10) */
    int32_t mdt_override;  /* > 0: use this MDT instead of the histogram (0) */
    int32_t hp_threshold;  /* HP switches to WD below this list size (1024);
                              a negative value disables the switch */
    int32_t loop_mode;     /* 0: device-resident loop (CUDA graph with a
                              conditional WHILE node); 1: host loop with a
                              worklist-size readback per iteration, as in the
                              paper's drivers (0) */
    int32_t wd_tile;       /* largest WD tile in worklist edges: 256..32768,
                              a multiple of 256 (8192); each iteration uses
                              the smallest multiple of 256 up to this that
                              gives every CTA about two tiles */
    int32_t ctas_per_sm;   /* CTAs per SM the fixed relax grid is sized for;
                              0 = the occupancy limit */
    int32_t hp_mode;       /* HP form: 0 = the paper's sub-iterations (Sec.
                              III-C: every node relaxes at most MDT edges per
                              sub-iteration, unfinished nodes form the next
                              sub-list); 1 = one step per super-iteration
                              with the list's nodes binned by degree into
                              sub-worklists served by a thread (<= min(MDT,
                              thread_max) edges), a warp (<= hp_warp_max) or
                              the whole CTA (more) (0) */
    int32_t hp_warp_max;   /* binned forms (hp_mode 1, ns_mode 1): largest
                              entry a warp serves; larger entries go to the
                              CTA bin (4096) */
    int32_t ns_mode;       /* NS form: 0 = the paper's thread per granule
                              (Sec. III-B: a split node's ceil(d/MDT) runs of
                              at most MDT edges, one thread each); 1 = the
                              same granules served by a thread (<=
                              thread_max edges), a warp (<= hp_warp_max) or
                              the whole CTA (0) */
    int32_t thread_max;    /* binned forms: largest entry one thread serves,
                              1..1024 (32) */
    int32_t hp_depth;      /* HP hierarchy depth, 1..8 (1): the first
                              hp_depth lists of a super-iteration's chain
                              (the super list, its sub-list, ...) each get
                              their own MDT, the histogram MDT of the
                              remaining degrees of that list's entries (the
                              super list uses the graph's MDT); later
                              sub-lists keep the last one (Sec. III-C leaves
                              the depth of the hierarchy to the user) */
    int32_t small_edges;   /* WD: while the worklist has at most this many
                              edges, levels run inside one persistent launch
                              (one CTA per SM, a grid barrier between levels)
                              instead of a launch per level: high-diameter
                              graphs have thousands of such levels.
                              0..16777216; 0 = off (65536) */
    int32_t test_barrier_skip; /* test hook, 0 in normal use: 1 makes CTA 1 of
                              the small-list launch leave before its first
                              grid barrier, so the other CTAs' bounded waits
                              run out (2 s) and the query returns
                              LB_ERR_TIMEOUT with the device still usable */
    int32_t bitmap_place;  /* 0..7 (0): where the visited / queued bitmap
                              starts inside its allocation, in steps of
                              min(1 MiB, one bitmap half rounded up to 4
                              KiB).  The bitmap is small and read at random
                              by every SM, and on GB300 the time of a BFS
                              depends on where its lines fall (R-MAT scale
                              24: 1.80 to 1.94 ms per query over eight
                              placements); lb_autotune picks the fastest.
                              The allocation carries the 7 steps of slack. */
    int32_t reserved[2];
} lb_options;

/* Device bytes by structure (lb_mem_report).  "extra" is everything a
 * strategy allocates beyond the CSR arrays, per query workspace. */
typedef struct lb_mem_stats {
    int64_t csr_offsets;   /* 8 (n+1) */
    int64_t csr_cols;      /* 4 m */
    int64_t csr_weights;   /* 4 m, 0 for an unweighted graph */
    int64_t status;        /* level / dist working array, 4 n */
    int64_t visited;       /* two bitmaps of n bits (each rounded up to 16
                              bytes): BFS visited bits in the first; SSSP
                              "queued in this iteration" bits of even and
                              odd iterations in both */
    int64_t node_lists;    /* node worklists (two buffers: id, first edge,
                              edge prefix) */
    int64_t tile_starts;   /* WD/HP: worklist entry holding every 256th
                              worklist edge (tile starts) */
    int64_t coo_src;       /* EP: COO source array (COO dst/wt are the CSR
                              cols/weights arrays, not duplicated) */
    int64_t edge_lists;    /* EP: edge worklists (two buffers of m ids) */
    int64_t sub_lists;     /* HP: sub-worklists (two buffers) */
    int64_t control;       /* counters, step trace */
    int64_t extra_total;   /* sum of the fields from status to control */
    int64_t base_total;    /* csr_offsets + csr_cols + csr_weights */
    int64_t resident;      /* bytes this graph holds on the device now */
    int64_t ns_children;   /* NS: child nodes created at the current MDT */
    int64_t mdt;           /* the MDT NS/HP use (0 if not yet computed) */
    int64_t ns_split;      /* NS_PHYS: child map, parent map and child
                              distances (4n + 8S); counted in extra_total */
} lb_mem_stats;

/* Per-query counters of the last query on a graph (lb_last_stats). */
typedef struct lb_query_stats {
    int64_t iterations;    /* worklist (super-)iterations */
    int64_t steps;         /* kernel steps (HP sub-iterations counted) */
    int64_t edges_relaxed; /* edge relaxations executed */
    int64_t pushes;        /* worklist entries pushed */
    int64_t mdt;           /* MDT used (NS/HP), else 0 */
    int32_t status;        /* lb_status of the query */
    int32_t strategy;      /* strategy that ran */
    double  device_ms;     /* GPU time of the query (events around it) */
} lb_query_stats;

/* One kernel step of the last query (lb_last_trace). */
typedef struct lb_step_record {
    int32_t level;         /* super-iteration (BFS level of the list) */
    int32_t mode;          /* 0 relax, 1 HP sub-iteration, 2 HP WD step,
                              3 HP degree-binned step (hp_mode 1), 4 WD
                              level inside the persistent small-list
                              launch */
    int64_t list_size;     /* entries in the list this step consumed */
    int64_t edges;         /* edges relaxed by this step */
    int64_t t_ns;          /* device time at the end of the step, in ns from
                              the start of the query (the set-up kernel) */
} lb_step_record;

/* ------------------------------------------------------------ graphs --- */

/* Copies a CSR graph to the device.  offsets: n+1 int64, offsets[0] = 0,
 * non-decreasing, offsets[n] = m; cols: m int32 in [0, n); weights: m
 * uint32 or NULL (BFS only).  Requires 1 <= n < 2^31 and m < 2^31.  The
 * caller keeps ownership of its arrays.  Errors: LB_ERR_ARG (validation),
 * LB_ERR_OOM, LB_ERR_CUDA. */
lb_status lb_graph_create(const int64_t *offsets, const int32_t *cols, const uint32_t *weights, int64_t n,
                          int64_t m, lb_graph **out);

/* Same, from device arrays already on the current device (copied; the
 * caller keeps ownership).  Only n and the ranges' sizes are checked on the
 * host; the CSR shape is validated on the device. */
lb_status lb_graph_create_dev(const int64_t *offsets_dev, const int32_t *cols_dev, const uint32_t *weights_dev,
                              int64_t n, int64_t m, lb_graph **out);

/* Frees every device allocation of the graph.  NULL is accepted. */
lb_status lb_graph_destroy(lb_graph *g);

lb_status lb_graph_info(const lb_graph *g, int64_t *n, int64_t *m, int32_t *weighted, int32_t *device);

/* Replaces the graph's options; cached device loops are rebuilt lazily. */
lb_status lb_set_options(lb_graph *g, const lb_options *o);
lb_status lb_get_options(const lb_graph *g, lb_options *o);

/* ----------------------------------------------------------- queries --- */

/* BFS from src.  levels_out: host array of n int32 receiving hop counts, -1
 * for unreachable vertices.  Blocks until the result is on the host. */
lb_status lb_bfs(lb_graph *g, int32_t src, lb_strategy s, int32_t *levels_out);

/* SSSP from src.  dist_out: host array of n uint32 receiving shortest
 * distances, 0xFFFFFFFF for unreachable vertices; a distance >= 2^32 - 2 is
 * written as 0xFFFFFFFE and the call returns LB_ERR_OVERFLOW.  Requires a
 * weighted graph (LB_ERR_UNSUPPORTED otherwise). */
lb_status lb_sssp(lb_graph *g, int32_t src, lb_strategy s, uint32_t *dist_out);

/* k host-output queries from srcs[0..k-1] (the paper's problem statement,
 * as for lb_bfs / lb_sssp, once per source).  out: host array of k * n
 * elements; the result of query i goes to out[i * n .. i * n + n - 1] (same
 * values and conventions as lb_bfs / lb_sssp).  Query i + 1 runs on the
 * device while the result of query i is copied to the host: the results
 * alternate between two device buffers of n words (the second one is held
 * with the workspaces until lb_release_workspaces) and the copies run on a
 * stream of their own, so with pinned host memory (cudaMallocHost or
 * cudaHostRegister) the copies overlap the traversals; with pageable memory
 * the results are the same but the copies serialise.  Every source is
 * checked before anything runs (LB_ERR_ARG).  The call returns once every
 * result is on the host, with LB_OK or the status of the first query that
 * failed (lb_last_error names it; SSSP: LB_ERR_OVERFLOW as in lb_sssp, the
 * other results still written).  lb_last_stats / lb_last_trace then
 * describe the last query.  k = 0 does nothing. */
lb_status lb_bfs_batch(lb_graph *g, const int32_t *srcs, int64_t k, lb_strategy s, int32_t *levels_out);
lb_status lb_sssp_batch(lb_graph *g, const int32_t *srcs, int64_t k, lb_strategy s, uint32_t *dist_out);

/* Device-output forms.  out_dev: n int32 (BFS levels) or n uint32 (SSSP
 * distances) on the graph's device; parents_dev: NULL or n int32 receiving
 * a shortest-path tree (parent[src] = src, -1 unreachable; the parent of v
 * is a u with an edge u->v and dist[u] + w(u,v) = dist[v]).  The call is
 * asynchronous on `stream`; its status is read with lb_last_stats(). */
lb_status lb_bfs_dev(lb_graph *g, int32_t src, lb_strategy s, int32_t *out_dev, int32_t *parents_dev, void *stream);
lb_status lb_sssp_dev(lb_graph *g, int32_t src, lb_strategy s, uint32_t *out_dev, int32_t *parents_dev,
                      void *stream);

/* Counters and status of the last query on g (waits for it to finish). */
lb_status lb_last_stats(lb_graph *g, lb_query_stats *out);

/* Per-step schedule of the last query: up to cap records, *len receives the
 * number of steps recorded (at most 4096 are kept). */
lb_status lb_last_trace(lb_graph *g, lb_step_record *out, int64_t cap, int64_t *len);

/* ----------------------------------------------------------- memory --- */

/* Device bytes a query with strategy s needs on g, by structure (the
 * paper's memory axis: Sec. II-B's COO cost 2E / 3E elements vs N + E for
 * CSR, and Sec. III's per-strategy extra space).  Pure arithmetic on n, m
 * and the options, except ns_children / mdt, which need the MDT (computed
 * on the device on first use). */
lb_status lb_mem_report(lb_graph *g, lb_strategy s, lb_mem_stats *out);

/* Releases every query workspace of g (the CSR stays). */
lb_status lb_release_workspaces(lb_graph *g);

/* Autotuner: times strategy s from each of the nsrc sources (kind
 * LB_KIND_BFS, LB_KIND_SSSP, or 2 for one BFS and one SSSP per source) under
 * a grid of options, keeps the fastest on g and returns it in *best with its
 * mean time per source in *best_ms (either may be NULL).  The grid per
 * strategy: WD -- the largest tile (2048..16384 edges) x CTAs per SM (the
 * occupancy limit, 2, 3, 4); HP -- the paper's sub-iterations with switch
 * threshold 256 / 1024 / 4096 x hierarchy depth 1..3, and the binned form
 * with threshold 256 / 1024 x thread bin 8 / 32 / 128 x warp bin 512 /
 * 4096 edges; NS -- the granule size (MDT from the histogram, or 32 / 256 /
 * 2048) in the paper's form, and the binned form with the histogram MDT or
 * 256 / 2048 x thread bin 8 / 32 / 128; NS_PHYS -- the granule size; BS, EP
 * -- CTAs per SM, each timed once.  Then, for WD, small_edges 0 (no
 * persistent small-list launch and no conditional node for it) against the
 * fastest grid option, and the eight bitmap placements (bitmap_place) of
 * each of the three fastest grid options.  Wherever the final choice is
 * made, the three fastest candidates are timed twice more and ranked by
 * the sum of their timings.  Fields outside the grid keep their values.
 * On any failure the options in force before the call are restored. */
lb_status lb_autotune(lb_graph *g, int32_t kind, lb_strategy s, const int32_t *srcs, int32_t nsrc, lb_options *best,
                      double *best_ms);

/* ------------------------------------------ schedule artefacts --- */

/* Histogram MDT (Sec. III-B, "Automatic Determination of Node Splitting
 * Threshold") of g's out-degrees, computed on the device: `bins`
 * equal-width bins over (0, maxDeg], bin k (1-based) holding degrees d with
 * (k-1) maxDeg < d bins <= k maxDeg; binIndex = tallest bin (smallest on a
 * tie); MDT = max(1, floor(binIndex maxDeg / bins)); 0 when g has no edges.
 * bins in [1, 4096].  Any output pointer may be NULL. */
lb_status lb_mdt(lb_graph *g, int32_t bins, int64_t *mdt, int64_t *max_degree, int32_t *bin_index);

/* Workload-decomposition start offsets (Sec. III-A) for a worklist whose F
 * nodes have out-degrees deg[] (host), cut over T threads: runs the
 * library's device worklist-push and tile-start code with
 * edgesPerThread = ceil(sum(deg) / T).  node_off[t], edge_off[t] (host, T
 * entries each) receive thread t's first worklist entry and the position of
 * its first edge inside that entry; threads past the last edge get (F, 0).
 * *ept receives edgesPerThread.  Uses the current device; F, T <= 2^24. */
lb_status lb_wd_offsets(const int64_t *deg, int64_t F, int64_t T, int64_t *node_off, int64_t *edge_off,
                        int64_t *ept);

/* ---------------------------------------------- batching / serving --- */

/* Many BFS / SSSP queries over many resident graphs run in one persistent
 * kernel (the paper runs one query at a time; batching is an addition).
 * Each query in flight owns a slot (its own worklists, bitmap, stamps and
 * loop state); the kernel's CTAs claim workload-decomposition tiles
 * (Sec. III-A) of any slot's current iteration, so iterations of different
 * queries interleave and finished slots take new requests at once
 * (continuous batching).  Results equal the single-query calls exactly. */
typedef struct lb_server lb_server;

typedef struct lb_server_options {
    int32_t slots;        /* queries in flight at most (0 = 256, at most
                             4096); how many run at once is also bounded by
                             the workspace pool (mem_fraction) */
    int32_t ctas_per_sm;  /* persistent grid: CTAs per SM (0 = occupancy) */
    int32_t tile;         /* largest work tile in worklist edges, 256..8192
                             (0 = 8192); a job's tiles shrink to spread it
                             over its share of the grid */
    int32_t idle_us;      /* the kernel exits after this long with no work
                             (0 = 1000); it is relaunched on demand */
    double mem_fraction;  /* share of free HBM the workspace pool may take,
                             reserved at creation; the pool is no larger
                             than `slots` queries on the largest graph need
                             (0 = 0.5).  Admission by memory: a query's
                             workspace (bitmaps and two worklists sized for
                             its own graph) is reserved in the pool when it
                             is admitted and returned when it completes; a
                             query that does not fit waits, in arrival
                             order, until completions free enough */
    int32_t launch_ms;    /* one persistent launch leaves after this long
                             (0 = 600000, ten minutes); while queries are
                             pending or in flight the next submit / poll
                             relaunches it and they continue where they
                             were (their state is in device memory) */
    int32_t policy;       /* tile claiming: 0 = the oldest query in flight
                             first (its iterations run as if it were alone;
                             the other queries fill the CTAs it leaves
                             idle), then round robin over the busy slots;
                             1 = round robin only (0) */
    int32_t items;        /* edges per thread per round in a RELAX tile: 2
                             or 3 (0 = 2) */
    int32_t reserved[5];
} lb_server_options;

typedef struct lb_server_info_t {
    int32_t slots;            /* queries in flight at most */
    int32_t grid;             /* CTAs of the persistent kernel */
    int64_t slot_bytes;       /* workspace bytes of a query on the largest graph */
    int64_t slot_n;           /* largest vertex count of a resident graph */
    int64_t kernel_launches;  /* persistent-kernel launches so far */
    int64_t submitted;
    int64_t completed;        /* completions returned by lb_server_poll */
    int64_t pool_bytes;       /* device memory pool for query workspaces */
    int64_t pool_free;        /* bytes of the pool not reserved now */
    int64_t pending;          /* submitted queries waiting for pool memory */
} lb_server_info_t;

typedef struct lb_completion {
    uint64_t ticket;          /* from lb_server_submit */
    int32_t status;           /* lb_status of the query */
    int32_t graph;
    int64_t iterations;       /* worklist iterations */
    int64_t edges_relaxed;
    int64_t device_ns;        /* admission to completion on the device */
} lb_completion;

/* graphs: ngraphs handles on the current device; they must outlive the
 * server.  Slot workspaces are sized for the largest graph. */
lb_status lb_server_create(lb_graph *const *graphs, int32_t ngraphs, const lb_server_options *opt,
                           lb_server **out);
lb_status lb_server_destroy(lb_server *s);
lb_status lb_server_info(const lb_server *s, lb_server_info_t *info);

/* Queues one query (non-blocking).  kind: LB_KIND_BFS / LB_KIND_SSSP;
 * out_dev: n int32 / uint32 on the device, written when the query
 * completes.  *ticket identifies its completion.  Fails with
 * LB_ERR_UNSUPPORTED when 65536 queries are outstanding (poll first). */
lb_status lb_server_submit(lb_server *s, int32_t graph, int32_t src, int32_t kind, void *out_dev, uint64_t *ticket);

/* Returns up to cap completed queries (non-blocking), in completion order,
 * and relaunches the persistent kernel if work is pending and it has left. */
lb_status lb_server_poll(lb_server *s, lb_completion *out, int32_t cap, int32_t *ndone);

/* Diagnostic snapshot of the engine (read while it runs): host and device
 * counters, and the first 16 busy slots with their current job. */
typedef struct lb_slot_state_t {
    int32_t slot, graph, kind, level;
    int32_t job_kind;   /* 0 none, 1 reset, 2 relax, 3 overflow check */
    int32_t job_tiles, job_done, job_gen;
    int64_t claim;      /* generation << 32 | next tile */
    int64_t in_cnt, in_edges;
    int32_t error, pad;
    int64_t ticket;
} lb_slot_state_t;

typedef struct lb_server_state_t {
    int64_t submitted, consumed, completed, acked;
    int32_t active, stopping, admit_lock, kernel_error;
    int32_t kernel_running, busy_slots, listed, pad;
    int64_t prof[8];    /* per-phase cycle counters of a profiling build, else 0 */
    lb_slot_state_t slot[16];
} lb_server_state_t;

lb_status lb_server_state(lb_server *s, lb_server_state_t *out);

/* Autotuner of the serving engine: runs the nreq sample requests (graph
 * index, source, kind; 1..4096 of them) as one batch on a server built with
 * each candidate of a grid of options -- edges per lane 2 / 3, CTAs per SM
 * (the occupancy limit / 3), largest tile 4096 / 8192 edges, claiming
 * policy 0 / 1 -- and returns in *best the candidate with the most
 * queries/s (second run of each; the first warms up), with that rate in
 * *best_qps (either may be NULL).  Fields outside the grid come from *base
 * (NULL: the defaults).  The sample's results go to device buffers the call
 * allocates and frees; the graphs are only read. */
lb_status lb_server_autotune(lb_graph *const *graphs, int32_t ngraphs, const lb_server_options *base,
                             const int32_t *req_graph, const int32_t *req_src, const int32_t *req_kind, int32_t nreq,
                             lb_server_options *best, double *best_qps);

/* Asks the persistent kernel to leave and waits for it (queries in flight
 * stay in their slots and resume at the next submit / poll). */
lb_status lb_server_stop(lb_server *s);

/* ------------------------------------------------- no allocation --- */

/* BFS with the workload-decomposition kernel for callers that cannot
 * allocate device memory (the paper has no counterpart: it is an
 * integration form).  Such callers include a process whose GPU memory is
 * entirely owned by another allocator, such as a framework's caching pool,
 * and a latency-bound service that must not call cudaMalloc once running,
 * because cudaMalloc can block and synchronise the device.
 *
 * offsets_dev (n+1 int64), cols_dev (m int32) and levels_dev (n int32,
 * receives hop counts, -1 unreachable) are caller-owned device pointers on
 * the current device; no lb_graph is used.  The CSR is checked on the
 * device before the traversal (offsets[0] = 0, non-decreasing, offsets[n] =
 * m, every column in [0, n)); a malformed one returns LB_ERR_ARG and
 * nothing else runs.  All other memory comes from one fixed array of device
 * memory inside the library (about 3.6 MiB; every GPU that loads the
 * library holds it until the process exits), so the call allocates
 * nothing.  Limits: n <= 131072
 * and m <= 16777216; larger sizes return LB_ERR_ARG.  The first call on a
 * device looks the array up (cudaGetSymbolAddress) and should come before
 * any stream capture.  The address is kept for the life of the process: a
 * process that resets the device (cudaDeviceReset) must not call this
 * entry point on that device afterwards.  Every call shares the array; calls whose GPU work
 * overlaps race and give wrong results.  The call waits for its result on
 * `stream` (it reads the worklist size back every iteration). */
lb_status lb_bfs_wd_noalloc(const int64_t *offsets_dev, const int32_t *cols_dev, int64_t n, int64_t m, int32_t src,
                            int32_t *levels_dev, void *stream);

/* ------------------------------------------------------------- misc --- */

/* Device allocator hook used for every later allocation (NULL, NULL
 * restores cudaMalloc / cudaFree).  alloc(bytes, ctx) returns a device
 * pointer or NULL; free(ptr, ctx).  Set it before creating graphs. */
lb_status lb_set_allocator(void *(*alloc_fn)(size_t, void *), void (*free_fn)(void *, void *), void *ctx);

/* Message describing the last error on the calling thread ("" if none). */
const char *lb_last_error(void);

/* Library version string. */
const char *lb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
