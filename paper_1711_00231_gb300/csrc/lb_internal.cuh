// Internal types shared by the host API and the device kernels of liblb.
//
// Data layout in HBM (one query workspace per graph, reused by every query):
//   status[n]        uint32 level / distance, 0xFFFFFFFF = not reached
//   bitmap[2 W]      W = ceil(n/32) rounded up to a multiple of 4 words.
//                    BFS: words 0..W-1 are the visited bits (claimed with
//                    atomicOr).  SSSP: the two halves are the "queued in
//                    this iteration" bits of even and odd iterations; an
//                    iteration sets bits in its own half and clears the
//                    other one, which the next iteration uses
//   node lists x2    worklist entries {v, beg, scan: int32 each} plus
//                    tstart[] (first entry of every WD tile); double-buffered
//   sub lists x2     HP sub-worklists, same layout
//   edge lists x2    EP worklists of CSR edge ids (COO edge index = CSR index)
//   coo_src[m]       EP: source of every CSR edge
//   Ctl              loop state, counters and the step trace
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lb.h"

namespace lbk {

constexpr uint32_t kInf = 0xFFFFFFFFu;  // not reached
constexpr uint32_t kSat = 0xFFFFFFFEu;  // saturated distance (>= 2^32 - 2)
constexpr int kBlock = 256;             // threads per CTA of every step kernel
constexpr int kWarps = kBlock / 32;
constexpr int kTraceMax = 4096;
constexpr int kHistMax = 4096;  // largest HistogramBinCount
// The persistent small-list kernel takes over once this many consecutive
// levels have produced lists of at most small_edges edges: a high-diameter
// graph has thousands of such levels, a skewed graph only a few at its
// start and end, where entering the persistent launch costs more than it
// saves.
constexpr uint32_t kSmallAfter = 4;
// Tile starts are recorded every kTileGrain worklist edges; an iteration
// then cuts its list into tiles of q * kTileGrain edges, q chosen from the
// list's size so that small lists still spread over many CTAs.
constexpr int64_t kTileGrain = 256;  // a power of two: the flush divides by it with shifts (>> 8)

// error bits in Ctl::error
enum : uint32_t {
    kErrCapacity = 1u,   // a push would exceed a list's capacity (dropped)
    kErrIterCap = 2u,    // iteration / step cap reached
    kErrSaturated = 4u,  // some relaxation saturated at 2^32 - 2
    kErrShape = 8u,      // CSR validation failed (device-created graphs)
    kErrOverflow = 16u,  // a final distance is saturated (>= 2^32 - 2)
    kErrZeroWeight = 32u,  // validation: the graph has a zero-weight edge (not an error)
    kErrBounds = 64u,    // a list entry pointed outside the graph (access skipped)
    kErrDeadline = 128u, // the query exceeded its device-side time limit
};

// step modes recorded in the trace
enum : int32_t { kModeRelax = 0, kModeHpSub = 1, kModeHpWd = 2, kModeHpBin = 3, kModeSmall = 4 };

// which list an HP step reads
enum : uint32_t { kHpFromSuper = 0, kHpFromSub = 1 };

struct TraceRec {
    int32_t level;
    int32_t mode;
    int64_t list_size;
    int64_t edges;
    int64_t t_ns;  // device time at the end of the step, from the query's start
};

// The counters every flush or CTA updates with atomics (the output list
// reservation, the done count, the push count) each start a 128-byte line
// of their own, away from the loop state every CTA reads when it starts.
// Measured on R-MAT scale 24: BFS level 2 520 -> 482-492 us, SSSP 1% faster.
#ifndef LB_CTL_PAD
#define LB_CTL_PAD 1
#endif
#if LB_CTL_PAD
#define LB_CTL_ALIGN alignas(128)
#else
#define LB_CTL_ALIGN
#endif
struct Ctl {
    // query parameters (written by the prepare kernel)
    uint32_t *status;
    int32_t src;
    int32_t kind;  // 0 BFS, 1 SSSP
    // loop state
    uint32_t level;     // super-iteration index = BFS level of the input list
    uint32_t par;       // input node list = lists[par], output = lists[par ^ 1]
    uint32_t in_cnt;    // entries of the input list
    uint32_t hp_from;   // HP: input list is the super list or a sub list
    uint64_t in_edges;  // edges of the input list (sum of entry lengths)
    // the output counter every flush reserves from (a line of its own)
    LB_CTL_ALIGN unsigned long long out_pack;  // output list: (entries << 32) | edges
    unsigned long long sub_pack;  // HP sub-list output: (entries << 32) | edges
    uint32_t hp_kind;   // HP: next step is a sub-iteration (1), WD (2) or binned (3)
    uint32_t hp_sub;    // HP: sub-iteration index inside the super-iteration
    uint32_t hp_mdt;    // HP: edges per node in the next sub-iteration
    uint32_t hp_lvl;    // HP: position of the input list in the super-iteration's chain
    uint32_t hp_mdt_pending;  // HP: the input sub-list needs its own MDT (k_hp_mdt)
    uint32_t hp_pad;
    unsigned long long sub_maxdeg;  // HP: largest remaining degree pushed to the sub-list
    unsigned long long small_pack[3];  // small-list levels: output counters, level L uses L % 3
    uint32_t bar_count;     // small-list levels: CTAs arrived at the grid barrier
    uint32_t bar_gen;       // small-list levels: barrier generation
    uint32_t bar_stop;      // small-list levels: the releasing CTA saw the time limit pass
    uint32_t small_run;     // consecutive levels ending with a list of at most small_edges edges
    uint32_t sub_in;    // HP: sub list buffer read when hp_from == kHpFromSub
    LB_CTL_ALIGN uint32_t blocks_done;
    uint32_t active;    // loop condition
    uint32_t error;
    uint32_t max_levels;
    uint64_t max_steps;
    uint64_t step;
    uint64_t t_deadline;  // %globaltimer (ns) after which the loop stops
    uint64_t t_start;     // %globaltimer (ns) when the query was prepared
    unsigned long long relaxed;
    LB_CTL_ALIGN unsigned long long pushes;
    uint32_t trace_len;
    uint32_t pad;
    TraceRec trace[kTraceMax];
    uint32_t hp_hist[kHistMax];  // HP depth > 1: histogram of a sub-list (zero between uses)
};

struct GraphDev {
    const int64_t *off;
    const int32_t *col;
    const uint32_t *w;
    int64_t n;
    int64_t m;
};

// Worklist entries.  Edge indices and list prefixes are below m < 2^31, so
// they are stored in 32 bits (half the bytes, single-instruction shuffles).
struct NodeList {
    int32_t *v;
    int32_t *beg;     // first CSR edge of the entry
    int32_t *scan;    // exclusive prefix of entry lengths; scan[cnt] = total
    int32_t *tstart;  // tstart[k]: entry holding list edge k * tile
};

struct StepParams {
    GraphDev g;
    Ctl *ctl;
    NodeList lists[2];
    NodeList subs[2];
    int32_t *elist[2];
    const int32_t *coo_src;
    uint32_t *bitmap;            // 2 * bm_words words (see the layout above)
    int64_t bm_words;            // W: words per bitmap half, a multiple of 4
    const int32_t *child_first;  // NS_PHYS: first child id of a split node, -1 if not split
    const int32_t *parent_of;    // NS_PHYS: parent of child n + i
    uint32_t *child_dist;        // NS_PHYS: mirrored distance of child n + i
    int64_t n_children;          // NS_PHYS: children created at p.mdt
    int64_t list_cap;
    int64_t tile_cap;   // tile-start entries per list (one per kTileGrain edges)
    int64_t elist_cap;
    int32_t tile;       // largest tile (edges) an iteration may use
    int32_t mdt;
    int32_t hp_threshold;  // <= 0: never switch to WD
    int32_t hp_mode;       // 0: sub-iterations, 1: degree-binned steps
    int32_t hp_warp_max;   // binned forms: largest entry a warp serves
    int32_t thread_max;    // binned forms: largest entry a thread serves
    int32_t ns_mode;       // 0: thread per granule, 1: binned granules
    int32_t hp_depth;      // HP: lists of a super-iteration's chain with their own MDT
    int32_t hist_bins;     // HistogramBinCount of the MDT heuristic
    int32_t test_barrier_skip;  // test hook: CTA 1 of the small-list launch skips its first barrier
    int32_t strategy;
    int32_t use_cond;
    int32_t small_edges;   // WD: lists of at most this many edges run in the persistent small-list kernel (0: off)
    cudaGraphConditionalHandle cond;
    cudaGraphConditionalHandle cond_small;  // device loop: run the small-list kernel on the next pass
    int32_t use_cond_small;
    int32_t pad2;
};

// ---- launch entry points implemented by the strategy translation units --
cudaError_t launch_step(int strategy, bool sssp, const StepParams &p, int grid, cudaStream_t st);
int step_blocks_per_sm(int strategy, bool sssp, int ns_mode);
cudaError_t launch_prepare(const StepParams &p, int32_t src, uint32_t *status, int kind, uint32_t max_levels,
                           uint64_t max_steps, uint64_t time_limit_ns, cudaStream_t st);
cudaError_t launch_init(const StepParams &p, int grid, cudaStream_t st);
cudaError_t launch_hp_mdt(const StepParams &p, int grid, cudaStream_t st);
cudaError_t launch_small_levels(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int small_ctas_per_sm();
cudaError_t launch_finish_query(const StepParams &p, cudaStream_t st);
cudaError_t launch_coo_build(const GraphDev &g, int32_t *coo_src, cudaStream_t st);
cudaError_t launch_mdt(const GraphDev &g, int32_t bins, unsigned long long *scratch, int64_t *result,
                       cudaStream_t st);
cudaError_t launch_validate(const GraphDev &g, uint32_t *err, cudaStream_t st);
cudaError_t launch_ns_count(const GraphDev &g, int32_t mdt, unsigned long long *out, cudaStream_t st);
cudaError_t launch_ns_phys_build(const GraphDev &g, int32_t mdt, int32_t *child_first, int32_t *parent_of,
                                 unsigned long long *block_sums, cudaStream_t st);
cudaError_t launch_wd_offsets(const int64_t *deg, int64_t F, int64_t T, NodeList list, Ctl *ctl, int64_t *ept_out,
                              cudaStream_t st);
cudaError_t launch_parents(const StepParams &p, bool sssp, int32_t *parents, cudaStream_t st);

// Sets the message lb_last_error() returns on the calling thread.
void set_last_error(const char *msg);

// Device CSR arrays of a graph (for the serving engine's graph table).
void graph_device_arrays(const lb_graph *g, const int64_t **off, const int32_t **col, const uint32_t **w);

}  // namespace lbk
