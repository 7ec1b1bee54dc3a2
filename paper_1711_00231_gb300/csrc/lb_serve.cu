// Batched / served queries: one persistent kernel runs many BFS / SSSP
// queries over many resident graphs at once.
//
// Every query in flight owns a slot: its own worklists, visited / queued
// bitmaps and loop state.  A slot always has at most one open job (reset its
// output, relax one worklist iteration with workload-decomposition tiles,
// or check for overflow), cut into tiles.  The CTAs of the persistent grid
// scan the slots and claim tiles with one atomicAdd on the slot's claim word
// (generation << 32 | next tile); the CTA that finishes a job's last tile
// finalises it and opens the slot's next job, so iterations of different
// queries interleave freely on the GPU and no grid-wide barrier exists.
//
// Requests arrive through a ring in pinned, device-mapped host memory: the
// host writes a request and then bumps `submitted`; a CTA that wins the
// admission lock (CTAs without work on every pass, busy ones now and then)
// moves pending requests into free slots.  Completions go back through a
// second mapped ring (one record per query, published by a sequence number
// written last).  The kernel leaves when it has had nothing to do for
// idle_ns, when the host raises `stop`, or once its launch time limit has
// passed (no CTA claims a tile after it); the host relaunches it while work
// is pending or in flight, and the queries continue from the slots' state.
//
// All loads of data other CTAs write during the kernel (worklists, status,
// bitmaps) bypass L1 (ld.global.cg), because L1 is not coherent within a
// kernel and slots are reused.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lb_steps.cuh"

namespace lbk {
namespace srv {

constexpr uint32_t kRing = 1u << 16;         // request / completion ring entries
constexpr int64_t kInitChunk = 1 << 16;      // vertices reset per INIT tile
// CTAs per SM the kernel is compiled for (the register budget); the edges
// per thread per round in a RELAX tile (2 or 3) are a server option, one
// kernel instance each
// Deferred claims in the serving kernel's relax tiles (as in the WD step).
// Measured on the 32-graph serving mix: 746 -> 904 queries/s batched, p99
// at the Poisson rate 239 -> 208 ms.
#ifndef LB_SERVE_DEFER_CLAIM
#define LB_SERVE_DEFER_CLAIM 1
#endif
#ifndef LB_SERVE_MIN_BLOCKS
#define LB_SERVE_MIN_BLOCKS 4
#endif
constexpr int kMaxSlots = 4096;  // slot indices fit 12 bits (Shared::oldest)
constexpr uint64_t kAdmitPeriodNs = 50000;  // a busy CTA retries admission this often

// Slot scheduling: 1 = round robin (after a tile a CTA moves on to the next
// slot, except that the CTA that opened a slot's next job takes its first
// tile) plus admission by busy CTAs; 0 = a CTA keeps to the slot it last
// claimed from, and only CTAs without work admit requests.
#ifndef LB_SERVE_POLICY
#define LB_SERVE_POLICY 1
#endif

// Build with -DLB_SERVE_PROFILE=1 to count SM cycles per phase of the
// persistent loop (thread 0 of every CTA; summed when a CTA leaves):
// 0 scan + claim that found a tile, 1 loops without a tile (scan,
// admission, back-off), 2 tile body up to the block barrier, 3 done count
// and job finalisation, 4 admission by busy CTAs, 5 tiles, 6 jobs finished,
// 7 loops without a tile.
#ifndef LB_SERVE_PROFILE
#define LB_SERVE_PROFILE 0
#endif

// Completion of a tile: 0 = block barrier, then one device-scope fence by
// thread 0 before the done count (the pattern of a cooperative grid
// barrier: the barrier orders the block's stores before thread 0's fence);
// 1 = every thread fences its own stores before the barrier as well.
#ifndef LB_SERVE_TILE_FENCE
#define LB_SERVE_TILE_FENCE 0
#endif


enum : uint32_t { kJobNone = 0, kJobInit = 1, kJobRelax = 2, kJobCheck = 3 };

struct Req {
    int32_t graph;
    int32_t src;
    int32_t kind;
    int32_t pad;
    unsigned long long out;
    unsigned long long ticket;
    unsigned long long ws;  // the query's workspace in the pool (reserved by the host)
};

// A query's workspace (one block of the server's device pool, reserved by
// the host before the request enters the ring): the visited / queued
// bitmap halves and two worklists sized for its own graph (n vertices, m
// edges), each piece 256-byte aligned.
struct WsLayout {
    int64_t bmw;       // words per bitmap half (a multiple of 4)
    int64_t cap;       // worklist entries
    int64_t tcap;      // tile-start entries per list
    uint64_t list0;    // byte offset of list 0 (list 1 follows at list0 + list_bytes)
    uint64_t v, beg, scan, tstart;  // byte offsets inside a list
    uint64_t list_bytes;
    uint64_t total;
};
__host__ __device__ constexpr uint64_t al256(uint64_t x) { return (x + 255u) & ~(uint64_t)255u; }
__host__ __device__ inline WsLayout ws_layout(int64_t n, int64_t m) {
    WsLayout L;
    L.bmw = ((n + 31) / 32 + 3) / 4 * 4;
    L.cap = n;
    L.tcap = m / kTileGrain + 2;
    L.list0 = al256(8u * (uint64_t)L.bmw);
    L.v = 0;
    L.beg = al256(4u * (uint64_t)L.cap);
    L.scan = L.beg + al256(4u * (uint64_t)L.cap);
    L.tstart = L.scan + al256(4u * (uint64_t)(L.cap + 1));
    L.list_bytes = L.tstart + al256(4u * (uint64_t)L.tcap);
    L.total = L.list0 + 2u * L.list_bytes;
    return L;
}
__host__ __device__ inline NodeList ws_list(unsigned char *ws, const WsLayout &L, uint32_t b) {
    unsigned char *base = ws + L.list0 + (uint64_t)b * L.list_bytes;
    NodeList l;
    l.v = (int32_t *)(base + L.v);
    l.beg = (int32_t *)(base + L.beg);
    l.scan = (int32_t *)(base + L.scan);
    l.tstart = (int32_t *)(base + L.tstart);
    return l;
}

struct Done {
    unsigned long long ticket;
    int32_t status;
    int32_t graph;
    uint32_t iterations;
    uint32_t pad;
    unsigned long long t_admit_ns;
    unsigned long long t_done_ns;
    unsigned long long edges_relaxed;
    unsigned long long seq;  // written last: index + 1 once the record is complete
};

struct HostShared {
    unsigned long long submitted;  // host: requests written
    unsigned long long consumed;   // device: requests taken into slots
    uint32_t stop;                 // host: leave the kernel
    uint32_t pad;
    Req req[kRing];
    Done done[kRing];
};

// The open job is described by ONE 64-bit word, so that a claimer reads
// generation, kind, tile size and tile count in a single load: with separate
// fields a late claimer could pair an old generation with a new tile count
// and take a tile of the next job twice.
//   bits 63..32 generation, 31..30 kind, 29..24 q (RELAX tile = q * 256
//   edges, q <= 32), 23..0 tiles (RELAX tiles < 2^31 / 256, INIT and CHECK
//   tiles < 2^31 / 2^16)
__host__ __device__ constexpr unsigned long long job_word(uint32_t gen, uint32_t kind, uint32_t q, uint32_t tiles) {
    return (unsigned long long)gen << 32 | (unsigned long long)(kind & 3u) << 30 |
           (unsigned long long)(q & 63u) << 24 | (unsigned long long)(tiles & 0xFFFFFFu);
}
__host__ __device__ constexpr uint32_t job_gen(unsigned long long w) { return (uint32_t)(w >> 32); }
__host__ __device__ constexpr uint32_t job_kind(unsigned long long w) { return (uint32_t)(w >> 30) & 3u; }
__host__ __device__ constexpr uint32_t job_q(unsigned long long w) { return (uint32_t)(w >> 24) & 63u; }
__host__ __device__ constexpr uint32_t job_tiles(unsigned long long w) { return (uint32_t)w & 0xFFFFFFu; }

struct Slot {
    unsigned long long claim;  // generation << 32 | next tile
    unsigned long long job;    // job_word(generation, kind, q, tiles)
    uint32_t job_done;
    uint32_t busy;
    int32_t graph;
    int32_t src;
    int32_t kind;
    uint32_t level;
    uint32_t par;
    uint32_t in_cnt;
    uint32_t error;
    uint32_t pad;
    uint64_t in_edges;
    unsigned long long out_pack;
    unsigned long long relaxed;
    unsigned long long pushes;
    unsigned long long ticket;
    unsigned long long t_admit;
    uint32_t *status;
    unsigned char *ws;  // the query's workspace (ws_layout of its graph): set at admission
};

struct Shared {  // device-global control of the persistent kernel
    uint32_t admit_lock;
    uint32_t active;         // busy slots
    uint32_t stopping;
    uint32_t error;
    unsigned long long consumed;
    unsigned long long completed;
    unsigned long long kernel_t0;
    unsigned long long prof[8];  // per-phase cycle counters (LB_SERVE_PROFILE)
    // oldest query in flight, as ticket << 12 | slot (kNoOldest: unknown):
    // lowered at admission and by every scan that sees an older busy slot,
    // reset when that query completes
    unsigned long long oldest;
    uint32_t busy_mask[kMaxSlots / 32];  // bit s: slot s holds a query (a scan hint)
};
constexpr unsigned long long kNoOldest = ~0ull;
__host__ __device__ constexpr unsigned long long oldest_pack(unsigned long long ticket, uint32_t slot) {
    return ticket << 12 | (unsigned long long)slot;
}

struct Params {
    Slot *slots;
    int32_t nslots;
    int32_t ngraphs;
    const GraphDev *graphs;
    HostShared *host;  // device view of the mapped ring
    Shared *sh;
    int32_t tile;
    int32_t policy;     // 0: the oldest query's tiles first, then round robin; 1: round robin
    uint64_t idle_ns;
    uint64_t hard_ns;
};

// Tile size of a RELAX job: the job's share of the grid is the grid divided
// by the busy slots, so with many queries in flight each job gets fewer,
// longer tiles (less claiming and finalising per edge), and a query alone
// spreads over the whole grid.
__device__ __forceinline__ int64_t job_tile(const Params &P, int64_t edges) {
    const uint32_t busy = __ldcg(&P.sh->active);
    const int64_t share = busy > 1 ? max((int64_t)1, (int64_t)gridDim.x / (int64_t)busy) : (int64_t)gridDim.x;
    return iteration_tile(edges, share, P.tile);
}

// ---- coherent (L2) loads and system-scope accesses ------------------------

template <class T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_sys32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int64_t list_search_cg(const int32_t *scan, int64_t lo, int64_t hi, int64_t e) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldcg(scan + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool bfs_claim_cg(uint32_t *bitmap, uint32_t *status, int32_t v, uint32_t newlev) {
    const uint32_t word = (uint32_t)v >> 5, bit = 1u << ((uint32_t)v & 31u);
    if (__ldcg(bitmap + word) & bit) return false;
    if (atomicOr(&bitmap[word], bit) & bit) return false;
    status[v] = newlev;
    return true;
}

__device__ __forceinline__ bool sssp_relax_cg(uint32_t *status, uint32_t *q, int32_t v, uint32_t du, uint32_t w,
                                              uint32_t *err) {
    if (du == kInf) return false;
    const uint64_t a64 = (uint64_t)du + (uint64_t)w;
    const uint32_t alt = a64 >= kSat ? kSat : (uint32_t)a64;
    if (alt >= __ldcg(status + v)) return false;
    const uint32_t old = atomicMin(&status[v], alt);
    if (alt >= old) return false;
    if (alt == kSat) atomicOr(err, kErrSaturated);
    if (is_queued<true>(q, v)) return false;
    const uint32_t bit = 1u << ((uint32_t)v & 31u);
    return !(atomicOr(&q[(uint32_t)v >> 5], bit) & bit);
}

// Dynamic slot fields change between jobs and are written by other SMs, so
// they are read through a volatile view (no L1); the pointer fields are
// fixed at server creation.
struct SlotState {
    int32_t graph, src, kind;
    uint32_t level, par, in_cnt;
    uint64_t in_edges;
    uint32_t *status;
    unsigned char *ws;
};

__device__ __forceinline__ SlotState slot_state(const Slot *S) {
    const volatile Slot *V = S;
    SlotState t;
    t.graph = V->graph;
    t.src = V->src;
    t.kind = V->kind;
    t.level = V->level;
    t.par = V->par;
    t.in_cnt = V->in_cnt;
    t.in_edges = V->in_edges;
    t.status = V->status;
    t.ws = V->ws;
    return t;
}

// ---- jobs ------------------------------------------------------------------

// Opens the slot's next job (single thread).  Parameters are written before
// the claim word moves to the new generation.
__device__ void open_job(Slot *S, uint32_t kind, uint32_t tiles, uint32_t q = 1) {
    const unsigned long long w = atomicAdd(&S->claim, 0ull);
    const uint32_t gen = (uint32_t)(w >> 32) + 1u;
    S->job_done = 0;
    __threadfence();
    atomicExch(&S->job, job_word(gen, kind, q, tiles));
    __threadfence();
    atomicExch(&S->claim, (unsigned long long)gen << 32);
}

__device__ void complete_query(const Params &P, Slot *S, int32_t status_code) {
    const unsigned long long idx = atomicAdd(&P.sh->completed, 1ull);
    Done *d = &P.host->done[idx % kRing];
    const volatile Slot *V = S;
    d->ticket = V->ticket;
    d->status = status_code;
    d->graph = V->graph;
    d->iterations = V->level;
    d->t_admit_ns = V->t_admit;
    d->t_done_ns = global_ns();
    d->edges_relaxed = V->relaxed;
    __threadfence_system();
    st_release_sys(&d->seq, idx + 1ull);
    const unsigned long long jw = atomicAdd(&S->job, 0ull);
    atomicExch(&S->job, job_word(job_gen(jw), kJobNone, 0u, 0u));
    __threadfence();
    // the slot's bit leaves the busy mask before the slot is released, so a
    // later admission of the slot (which needs busy == 0) sets it again
    const uint32_t si = (uint32_t)(S - P.slots);
    atomicCAS(&P.sh->oldest, oldest_pack(V->ticket, si), kNoOldest);
    atomicAnd(&P.sh->busy_mask[si >> 5], ~(1u << (si & 31u)));
    __threadfence();
    S->busy = 0;
    atomicSub(&P.sh->active, 1u);
}

__device__ int32_t slot_status(const Slot *S) {
    const uint32_t e = ((const volatile Slot *)S)->error;
    if (e & (kErrCapacity | kErrShape | kErrBounds)) return LB_ERR_INTERNAL;
    if (e & (kErrIterCap | kErrDeadline)) return LB_ERR_TIMEOUT;
    if (e & kErrOverflow) return LB_ERR_OVERFLOW;
    return LB_OK;
}

// Finalises the slot's job after its last tile (single thread).  Returns
// true when the slot has a next job open.
__device__ bool finish_job(const Params &P, Slot *S, uint32_t kind) {
    const SlotState st = slot_state(S);
    const GraphDev g = P.graphs[st.graph];
    if (kind == kJobInit) {
        const int64_t beg = g.off[st.src];
        const int64_t deg = g.off[st.src + 1] - beg;
        S->level = 0;
        S->par = 0;
        S->out_pack = 0ull;
        S->relaxed = 0ull;
        if (deg == 0) {
            S->level = 1;
            complete_query(P, S, LB_OK);
            return false;
        }
        const WsLayout W = ws_layout(g.n, g.m);
        NodeList L = ws_list(st.ws, W, 0);
        L.v[0] = st.src;
        L.beg[0] = (int32_t)beg;
        L.scan[0] = 0;
        L.scan[1] = (int32_t)deg;
        const int64_t grains = (deg + kTileGrain - 1) / kTileGrain;
        for (int64_t k = 0; k < grains && k < W.tcap; ++k) L.tstart[k] = 0;
        S->in_cnt = 1;
        S->in_edges = (uint64_t)deg;
        const int64_t Tj = job_tile(P, deg);
        open_job(S, kJobRelax, (uint32_t)((deg + Tj - 1) / Tj), (uint32_t)(Tj / kTileGrain));
        return true;
    }
    if (kind == kJobRelax) {
        const unsigned long long pk = ld_volatile(&S->out_pack);
        int64_t cnt = (int64_t)(pk >> 32);
        const int64_t edges = (int64_t)(pk & 0xFFFFFFFFull);
        const WsLayout W = ws_layout(g.n, g.m);
        if (cnt > W.cap) { atomicOr(&S->error, kErrCapacity); cnt = W.cap; }
        S->relaxed = ld_volatile(&S->relaxed) + st.in_edges;
        S->level = st.level + 1;
        const uint32_t out = st.par ^ 1u;
        const uint32_t err = atomicOr(&S->error, 0u);
        if (cnt > 0 && st.level + 1 <= (uint32_t)g.n && !(err & (kErrCapacity | kErrBounds))) {
            ws_list(st.ws, W, out).scan[cnt] = (int32_t)edges;
            S->par = out;
            S->in_cnt = (uint32_t)cnt;
            S->in_edges = (uint64_t)edges;
            S->out_pack = 0ull;
            const int64_t Tj = job_tile(P, edges);
            open_job(S, kJobRelax, (uint32_t)((edges + Tj - 1) / Tj), (uint32_t)(Tj / kTileGrain));
            return true;
        }
        if (cnt > 0 && !(err & (kErrCapacity | kErrBounds))) atomicOr(&S->error, kErrIterCap);
        if (st.kind == 1 && (err & kErrSaturated)) {
            open_job(S, kJobCheck, (uint32_t)((g.n + kInitChunk - 1) / kInitChunk));
            return true;
        }
        complete_query(P, S, slot_status(S));
        return false;
    }
    complete_query(P, S, slot_status(S));  // kJobCheck
    return false;
}

// ---- tile bodies (block-wide) ------------------------------------------------

__device__ void init_tile(const Params &P, Slot *S, int64_t k) {
    const SlotState st = slot_state(S);
    const GraphDev g = P.graphs[st.graph];
    const int64_t v0 = k * kInitChunk;
    const int64_t v1 = min(v0 + kInitChunk, g.n);
    const int32_t src = st.src;
    const bool sssp = st.kind == 1;
    uint32_t *status = st.status;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) status[i] = i == src ? 0u : kInf;
    // BFS: this chunk's visited bits; SSSP: its queued bits in both halves
    // (kInitChunk is a multiple of 32, so chunks own whole words)
    const WsLayout W = ws_layout(g.n, g.m);
    uint32_t *bitmap = (uint32_t *)st.ws;
    const int64_t w0 = v0 / 32, w1 = (v1 + 31) / 32;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        bitmap[w] = (!sssp && w == (src >> 5)) ? (1u << (src & 31)) : 0u;
        if (sssp) bitmap[W.bmw + w] = 0u;
    }
}

__device__ void check_tile(const Params &P, Slot *S, int64_t k) {
    const SlotState st = slot_state(S);
    const GraphDev g = P.graphs[st.graph];
    const int64_t v0 = k * kInitChunk;
    const int64_t v1 = min(v0 + kInitChunk, g.n);
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x)
        if (__ldcg(st.status + i) == kSat) atomicOr(&S->error, kErrOverflow);
}

template <bool SSSP, int ITEMS>
__device__ void relax_tile(const Params &P, Slot *S, int64_t t, int64_t ntiles, int64_t q, WarpBuf &wb,
                           NoScratch &ws) {
    const SlotState st = slot_state(S);
    const GraphDev g = P.graphs[st.graph];
    const WsLayout W = ws_layout(g.n, g.m);
    uint32_t *bitmap = (uint32_t *)st.ws;
    uint32_t *qcur = queued_half(bitmap, W.bmw, st.level);
    if (SSSP) {
        // The other half still holds the bits of the previous iteration,
        // whose queued vertices are exactly this iteration's list entries
        // (a vertex without out-edges is queued but never listed; its stale
        // bit is harmless, as such a vertex is never listed or expanded).
        // Tile t clears the bits of its share of the entries for the next
        // iteration, which starts only after every tile of this one.
        uint32_t *qn = queued_half(bitmap, W.bmw, st.level + 1u);
        const int64_t per = ((int64_t)st.in_cnt + ntiles - 1) / ntiles;
        const int64_t k0 = t * per, k1 = min(k0 + per, (int64_t)st.in_cnt);
        const int32_t *vin = ws_list(st.ws, W, st.par).v;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const int32_t u = __ldcg(vin + k);
            if (u >= 0 && (int64_t)u < g.n) atomicAnd(&qn[(uint32_t)u >> 5], ~(1u << ((uint32_t)u & 31u)));
        }
    }
    FlushOut o;
    o.list = ws_list(st.ws, W, st.par ^ 1u);
    o.elist = nullptr;
    o.pack = &S->out_pack;
    o.cap = W.cap;
    o.tile_cap = W.tcap;
    o.tile = (int32_t)kTileGrain;
    o.mdt = 1;
    o.err = &S->error;
    o.pushes = &S->pushes;
    o.child_first = nullptr;
    o.off = g.off;
    o.defer = SSSP ? (LB_SERVE_DEFER_CLAIM ? 3 : LB_DEFER_OFFSETS) : (LB_SERVE_DEFER_CLAIM ? 2 : LB_DEFER_OFFSETS);
    o.claim_bitmap = SSSP ? qcur : bitmap;
    o.claim_status = st.status;
    o.claim_level = st.level;
    uint32_t cnt = 0;
    wd_walk_tile<SSSP, ITEMS, true>(g, ws_list(st.ws, W, st.par), st.in_cnt, (int64_t)st.in_edges, q * kTileGrain,
                                     t, bitmap, qcur, st.status, st.level, &S->error, wb, ws, cnt, o);
#if LB_BLOCK_FLUSH
    wflush_block<kOutNode, true>(wb, ws, cnt, o);
#else
    wflush<kOutNode, true>(wb, ws, cnt, o);
#endif
}

// ---- admission -------------------------------------------------------------

__device__ void admit(const Params &P) {
    Shared *sh = P.sh;
    const unsigned long long sub = ld_acquire_sys(&P.host->submitted);
    unsigned long long con = __ldcg(&sh->consumed);  // written by whichever CTA held the lock last
    int32_t cursor = 0;
    while (con < sub) {
        Slot *S = nullptr;
        for (; cursor < P.nslots; ++cursor)
            if (((volatile Slot *)&P.slots[cursor])->busy == 0) {
                S = &P.slots[cursor];
                break;
            }
        if (!S) break;
        const volatile Req *vr = &P.host->req[con % kRing];  // host memory, written by the host
        Req r;
        r.graph = vr->graph;
        r.src = vr->src;
        r.kind = vr->kind;
        r.out = vr->out;
        r.ticket = vr->ticket;
        r.ws = vr->ws;
        S->ticket = r.ticket;
        S->ws = reinterpret_cast<unsigned char *>(r.ws);
        S->graph = r.graph;
        S->src = r.src;
        S->kind = r.kind;
        S->status = reinterpret_cast<uint32_t *>(r.out);
        S->error = 0;
        S->t_admit = global_ns();
        S->level = 0;
        S->relaxed = 0ull;
        S->pushes = 0ull;
        S->out_pack = 0ull;
        bool valid = r.graph >= 0 && r.graph < P.ngraphs && r.out != 0ull && (r.kind == 0 || r.kind == 1);
        if (valid) {
            const GraphDev g = P.graphs[r.graph];
            valid = r.src >= 0 && (int64_t)r.src < g.n && r.ws != 0ull && (r.kind == 0 || g.w != nullptr);
        }
        S->busy = 1;
        atomicAdd(&sh->active, 1u);
        atomicOr(&sh->busy_mask[(uint32_t)cursor >> 5], 1u << ((uint32_t)cursor & 31u));
        if (valid) atomicMin(&sh->oldest, oldest_pack(r.ticket, (uint32_t)cursor));
        ++con;
        if (!valid) {
            complete_query(P, S, LB_ERR_ARG);
            continue;
        }
        const GraphDev g = P.graphs[r.graph];
        open_job(S, kJobInit, (uint32_t)((g.n + kInitChunk - 1) / kInitChunk));
    }
    sh->consumed = con;
    st_release_sys(&P.host->consumed, con);
}

// Takes the admission lock if free and, unless the grid is leaving, admits
// pending requests into free slots (thread 0 of a CTA).  Returns whether
// the lock was taken; *admitted tells whether any request was admitted.
__device__ bool try_admit(const Params &P, bool *admitted) {
    *admitted = false;
    if (atomicCAS(&P.sh->admit_lock, 0u, 1u) != 0u) return false;
    if (__ldcg(&P.sh->stopping) == 0u) {
        const unsigned long long before = __ldcg(&P.sh->consumed);
        admit(P);
        *admitted = __ldcg(&P.sh->consumed) != before;
    }
    return true;
}

__device__ void release_admit(const Params &P) {
    __threadfence();
    atomicExch(&P.sh->admit_lock, 0u);
}

// ---- the persistent kernel -------------------------------------------------

template <int ITEMS>
__global__ void __launch_bounds__(kBlock, LB_SERVE_MIN_BLOCKS) k_serve(Params P) {
    __shared__ WarpBuf s_wb[kWarps];
    NoScratch ns;  // node pushes only: no flush scratch
    __shared__ int s_slot;
    __shared__ uint32_t s_kind, s_tiles, s_q;
    __shared__ long long s_tile;
    __shared__ int s_exit;
    __shared__ uint32_t s_scan_from;
    const uint32_t warp = threadIdx.x >> 5;
    uint64_t idle_since = 0;
    uint64_t last_admit = 0;
#if LB_SERVE_PROFILE
    unsigned long long pf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long c_top = 0, c_mid = 0;
#define PF_MARK(v) (v) = clock64()
#define PF_ADD(i, v) pf[i] += (unsigned long long)((v))
#else
#define PF_MARK(v)
#define PF_ADD(i, v)
#endif
    if (threadIdx.x == 0) s_scan_from = blockIdx.x % (uint32_t)P.nslots;
    const uint64_t t_launch = __ldcg(&P.sh->kernel_t0);  // written by k_serve_t0 before this launch
    for (;;) {
        // every thread has read the previous iteration's s_* values before
        // thread 0 overwrites them (without this barrier a lagging warp could
        // pick up the next tile out of step with its block)
        __syncthreads();
        if (threadIdx.x == 0) PF_MARK(c_top);
        if (threadIdx.x < 32) {
            // warp 0 reads up to 32 words of the busy mask in one L2 round
            // trip, then for each word with busy slots (round robin from the
            // slot after the one it last worked on, which itself comes first
            // when this CTA just opened its next job) each lane reads one
            // slot's claim and job words, and the claimable slots are tried
            // in order until a claim holds
            const uint32_t lane = threadIdx.x;
            // past the launch's time limit a CTA claims nothing more and
            // leaves (checked before every claim: a CTA that keeps finding
            // work, such as the one that opens a slot's next job, would
            // otherwise never see the limit)
            int late = 0;
            if (lane == 0) late = global_ns() - t_launch > P.hard_ns;
            late = __shfl_sync(kFull, late, 0);
            const uint32_t scan_from = s_scan_from;
            uint32_t nw = late ? 0u : ((uint32_t)P.nslots + 31u) >> 5;
            const uint32_t sw = scan_from >> 5;
            int found = -1;
            uint32_t f_kind = 0, f_tiles = 0, f_tile = 0, f_q = 0;
            unsigned long long seen_oldest = kNoOldest;  // oldest busy slot this scan saw
            if (P.policy == 0 && !late) {
                // the oldest query in flight first: its iterations then run as
                // if it were alone, and the other queries fill the CTAs its
                // current iteration leaves idle
                int ok = 0;
                uint32_t k2 = 0, t2 = 0, q2 = 0, idx = 0, hs = 0;
                if (lane == 0) {
                    const unsigned long long op = __ldcg(&P.sh->oldest);
                    hs = (uint32_t)(op & 4095ull);
                    if (op != kNoOldest && hs < (uint32_t)P.nslots) {
                        Slot *S = &P.slots[hs];
                        const unsigned long long cw = __ldcg(&S->claim);
                        const unsigned long long jw = __ldcg(&S->job);
                        if (job_kind(jw) != kJobNone && job_gen(jw) == (uint32_t)(cw >> 32) &&
                            (uint32_t)cw < job_tiles(jw)) {
                            const unsigned long long old = atomicAdd(&S->claim, 1ull);
                            __threadfence();
                            const unsigned long long jw2 = atomicAdd(&S->job, 0ull);
                            k2 = job_kind(jw2);
                            t2 = job_tiles(jw2);
                            q2 = job_q(jw2);
                            idx = (uint32_t)old;
                            ok = job_gen(jw2) == (uint32_t)(old >> 32) && k2 != kJobNone && idx < t2;
                        }
                    }
                }
                if (__shfl_sync(kFull, ok, 0)) {
                    found = (int)__shfl_sync(kFull, hs, 0);
                    f_kind = __shfl_sync(kFull, k2, 0);
                    f_tiles = __shfl_sync(kFull, t2, 0);
                    f_q = __shfl_sync(kFull, q2, 0);
                    f_tile = __shfl_sync(kFull, idx, 0);
                    nw = 0u;
                }
            }
            for (uint32_t base = 0; base < nw && found < 0; base += 32) {
                uint32_t wmask = 0;
                if (base + lane < nw) wmask = __ldcg(&P.sh->busy_mask[(sw + base + lane) % nw]);
                unsigned nz = __ballot_sync(kFull, wmask != 0u);
                while (nz && found < 0) {
                    const int wl = __ffs(nz) - 1;
                    nz &= nz - 1;
                    const uint32_t w = (sw + base + (uint32_t)wl) % nw;
                    const uint32_t bits = __shfl_sync(kFull, wmask, wl);
                    const uint32_t rot = (base == 0 && wl == 0) ? (scan_from & 31u) : 0u;
                    const uint32_t sl = (lane + rot) & 31u;
                    const int32_t si = (int32_t)(32u * w + sl);
                    bool claimable = false;
                    unsigned long long mine = kNoOldest;
                    if (((bits >> sl) & 1u) && si < P.nslots) {
                        const Slot *S = &P.slots[si];
                        const unsigned long long cw = __ldcg(&S->claim);
                        const unsigned long long jw = __ldcg(&S->job);
                        claimable = job_kind(jw) != kJobNone && job_gen(jw) == (uint32_t)(cw >> 32) &&
                                    (uint32_t)cw < job_tiles(jw);
                        if (job_kind(jw) != kJobNone) mine = oldest_pack(__ldcg(&S->ticket), (uint32_t)si);
                    }
                    if (P.policy == 0) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const unsigned long long x = __shfl_xor_sync(kFull, mine, o);
                            mine = x < mine ? x : mine;
                        }
                        seen_oldest = mine < seen_oldest ? mine : seen_oldest;
                    }
                    unsigned cand = __ballot_sync(kFull, claimable);
                    while (cand) {
                        const int l = __ffs(cand) - 1;
                        cand &= cand - 1;
                        int ok = 0;
                        uint32_t k2 = 0, t2 = 0, q2 = 0, idx = 0;
                        if ((int)lane == l) {
                            Slot *S = &P.slots[si];
                            const unsigned long long old = atomicAdd(&S->claim, 1ull);
                            __threadfence();
                            // the claim counts only if the job word still belongs
                            // to the generation it was taken in (a late claim on a
                            // finished job must not take a tile of the next job)
                            const unsigned long long jw = atomicAdd(&S->job, 0ull);
                            k2 = job_kind(jw);
                            t2 = job_tiles(jw);
                            q2 = job_q(jw);
                            idx = (uint32_t)old;
                            ok = job_gen(jw) == (uint32_t)(old >> 32) && k2 != kJobNone && idx < t2;
                        }
                        ok = __shfl_sync(kFull, ok, l);
                        if (ok) {
                            found = __shfl_sync(kFull, si, l);
                            f_kind = __shfl_sync(kFull, k2, l);
                            f_tiles = __shfl_sync(kFull, t2, l);
                            f_q = __shfl_sync(kFull, q2, l);
                            f_tile = __shfl_sync(kFull, idx, l);
                            break;
                        }
                    }
                }
            }
            if (lane == 0) {
                // the hint catches up with the oldest busy slot any scan sees
                if (seen_oldest != kNoOldest && seen_oldest < __ldcg(&P.sh->oldest))
                    atomicMin(&P.sh->oldest, seen_oldest);
                if (found >= 0) s_scan_from = (uint32_t)found;
                s_slot = found;
                s_exit = late;
                if (late) atomicOr(&P.sh->error, kErrDeadline);
                if (found >= 0) {
                    s_kind = f_kind;
                    s_tiles = f_tiles;
                    s_q = f_q;
                    s_tile = (long long)f_tile;
                }
            }
        }
        if (threadIdx.x == 0) {
            if (s_slot < 0 && !s_exit) {
                const uint64_t now = global_ns();
                // Admission and the decision to stop are taken under one lock,
                // so no request is admitted after the grid decided to leave.
                bool admitted = false;
                if (try_admit(P, &admitted)) {
                    last_admit = now;
                    if (__ldcg(&P.sh->stopping) == 0u) {
                        if (admitted || __ldcg(&P.sh->active) != 0u) {
                            idle_since = 0;
                        } else if (idle_since == 0) {
                            idle_since = now;
                        } else if (now - idle_since > P.idle_ns) {
                            atomicExch(&P.sh->stopping, 1u);
                        }
                    }
                    release_admit(P);
                }
                if (ld_acquire_sys32(&P.host->stop) != 0u || __ldcg(&P.sh->stopping) != 0u) s_exit = 1;
                if (!s_exit) __nanosleep(256);
            } else if (s_slot >= 0) {
                idle_since = 0;
            }
        }
        __syncthreads();
#if LB_SERVE_PROFILE
        if (threadIdx.x == 0) {
            PF_MARK(c_mid);
            if (s_slot >= 0) PF_ADD(0, c_mid - c_top);
            else { PF_ADD(1, c_mid - c_top); PF_ADD(7, 1); }
        }
        if (s_exit) {
            if (threadIdx.x == 0)
                for (int i = 0; i < 8; ++i) atomicAdd(&P.sh->prof[i], pf[i]);
            break;
        }
#else
        if (s_exit) break;
#endif
        const int si = s_slot;
        if (si < 0) continue;
        Slot *S = &P.slots[si];
        const uint32_t kind = s_kind;
        if (kind == kJobInit) init_tile(P, S, s_tile);
        else if (kind == kJobCheck) check_tile(P, S, s_tile);
        else if (((const volatile Slot *)S)->kind == 1)
            relax_tile<true, ITEMS>(P, S, s_tile, s_tiles, s_q, s_wb[warp], ns);
        else relax_tile<false, ITEMS>(P, S, s_tile, s_tiles, s_q, s_wb[warp], ns);
        // Other CTAs read this tile's stores (list entries, resets) in the
        // slot's next job within this same kernel: they are made visible
        // device-wide before the tile is counted as done.
#if LB_SERVE_TILE_FENCE
        __threadfence();
#endif
        __syncthreads();
        if (threadIdx.x == 0) {
#if LB_SERVE_PROFILE
            long long c_b = clock64();
            PF_ADD(2, c_b - c_mid);
            PF_ADD(5, 1);
#endif
            __threadfence();
            const uint32_t d = atomicAdd(&S->job_done, 1u);
            bool reopened = false;
            if (d == s_tiles - 1) {
                __threadfence();
                reopened = finish_job(P, S, kind);
                PF_ADD(6, 1);
            }
#if LB_SERVE_PROFILE
            long long c_d = clock64();
            PF_ADD(3, c_d - c_b);
#endif
#if LB_SERVE_POLICY == 1
            // round robin, except that the CTA which opened the slot's next
            // job takes its first tile (a query's chain of small iterations
            // then runs without waiting for a scan to come by)
            s_scan_from = reopened ? (uint32_t)si : ((uint32_t)si + 1u) % (uint32_t)P.nslots;
            // busy CTAs also refill free slots, so that admission does not
            // wait until some CTA runs out of work
            const uint64_t now = global_ns();
            if (now - last_admit > kAdmitPeriodNs && __ldcg(&P.sh->active) < (uint32_t)P.nslots) {
                last_admit = now;
                bool admitted = false;
                if (try_admit(P, &admitted)) release_admit(P);
            }
#if LB_SERVE_PROFILE
            PF_ADD(4, clock64() - c_d);
#endif
#else
            (void)reopened;
            (void)last_admit;
#endif
        }
    }
}

__global__ void k_serve_t0(Shared *sh) {
    sh->kernel_t0 = global_ns();
    sh->stopping = 0;
    sh->admit_lock = 0;
}

}  // namespace srv
}  // namespace lbk

// =========================================================================
// host side
// =========================================================================

using namespace lbk;
using namespace lbk::srv;

struct lb_server {
    int device = 0;
    int sms = 0;
    std::mutex mu;
    lb_server_options opt{};
    std::vector<lb_graph *> graphs;
    std::vector<int64_t> graph_n, graph_m;
    std::vector<bool> graph_weighted;
    GraphDev *d_graphs = nullptr;
    Slot *d_slots = nullptr;
    Shared *d_shared = nullptr;
    HostShared *h_ring = nullptr;  // pinned, mapped
    HostShared *d_ring = nullptr;  // device view
    int32_t nslots = 0;
    int64_t slot_n = 0;            // largest vertex count of a resident graph
    int64_t slot_bytes = 0;        // workspace bytes of a query on the largest graph
    // Admission by device memory: every query's workspace is a block of
    // this pool, reserved on the host (first fit, free neighbours merged)
    // before its request enters the device ring; a request that does not
    // fit waits in `pending` (arrival order) until completions free memory.
    unsigned char *pool = nullptr;
    uint64_t pool_bytes = 0, pool_free = 0;
    std::map<uint64_t, uint64_t> free_ranges;  // offset -> bytes
    std::unordered_map<unsigned long long, std::pair<uint64_t, uint64_t>> held;  // ticket -> (offset, bytes)
    struct Pending {
        int32_t graph, src, kind;
        unsigned long long out, ticket;
        uint64_t bytes;
    };
    std::deque<Pending> pending;
    int grid = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_kernel = nullptr;
    bool launched = false;
    unsigned long long submitted = 0;  // host copy
    unsigned long long acked = 0;      // completions handed to the caller
    unsigned long long next_ticket = 1;
    uint64_t launches = 0;
};

namespace {

lb_status sfail(lb_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[384];
    if (e != cudaSuccess) snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof(buf), "%s", msg);
    set_last_error(buf);
    return s;
}

#define SV_CU(call, what)                                                    \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return sfail(e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, what, e_); \
    } while (0)

// First fit in the pool; every block is a multiple of 256 bytes.
bool pool_alloc(lb_server *s, uint64_t bytes, uint64_t *off) {
    for (auto it = s->free_ranges.begin(); it != s->free_ranges.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const uint64_t rest = it->second - bytes, at = it->first + bytes;
        s->free_ranges.erase(it);
        if (rest) s->free_ranges[at] = rest;
        s->pool_free -= bytes;
        return true;
    }
    return false;
}

void pool_release(lb_server *s, uint64_t off, uint64_t bytes) {
    auto it = s->free_ranges.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_ranges.end() && it->first + it->second == nx->first) {  // merge with the next range
        it->second += nx->second;
        s->free_ranges.erase(nx);
    }
    if (it != s->free_ranges.begin()) {  // and with the previous one
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_ranges.erase(it);
        }
    }
    s->pool_free += bytes;
}

uint64_t query_bytes(const lb_server *s, int32_t graph) {
    const WsLayout L = ws_layout(s->graph_n[(size_t)graph], s->graph_m[(size_t)graph]);
    return al256(L.total);
}

// Moves pending requests, in arrival order, into the device ring while
// their workspaces fit in the pool (the first that does not fit waits, so
// a large query is not overtaken forever by smaller ones).
void pump(lb_server *s) {
    bool moved = false;
    while (!s->pending.empty() && s->submitted - s->acked < kRing) {
        const lb_server::Pending &q = s->pending.front();
        uint64_t off = 0;
        if (!pool_alloc(s, q.bytes, &off)) break;
        Req &r = s->h_ring->req[s->submitted % kRing];
        r.graph = q.graph;
        r.src = q.src;
        r.kind = q.kind;
        r.out = q.out;
        r.ticket = q.ticket;
        r.ws = (unsigned long long)(uintptr_t)(s->pool + off);
        s->held[q.ticket] = {off, q.bytes};
        s->submitted++;
        s->pending.pop_front();
        moved = true;
    }
    if (moved) __atomic_store_n(&s->h_ring->submitted, s->submitted, __ATOMIC_RELEASE);
}

void destroy_server(lb_server *s) {
    if (!s) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (s->h_ring) {
        __atomic_store_n(&s->h_ring->stop, 1u, __ATOMIC_RELEASE);
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->pool) cudaFree(s->pool);
    if (s->d_graphs) cudaFree(s->d_graphs);
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->d_shared) cudaFree(s->d_shared);
    if (s->h_ring) cudaFreeHost(s->h_ring);
    if (s->ev_kernel) cudaEventDestroy(s->ev_kernel);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

bool kernel_running(lb_server *s) {
    if (!s->launched) return false;
    const cudaError_t q = cudaEventQuery(s->ev_kernel);
    if (q == cudaErrorNotReady) return true;
    s->launched = false;
    return false;
}

lb_status launch_kernel(lb_server *s) {
    Params P;
    memset(&P, 0, sizeof(P));
    P.slots = s->d_slots;
    P.nslots = s->nslots;
    P.ngraphs = (int32_t)s->graphs.size();
    P.graphs = s->d_graphs;
    P.host = s->d_ring;
    P.sh = s->d_shared;
    P.tile = s->opt.tile;
    P.policy = s->opt.policy;
    P.idle_ns = (uint64_t)s->opt.idle_us * 1000ull;
    P.hard_ns = (uint64_t)s->opt.launch_ms * 1000000ull;  // one persistent launch never outlives this
    k_serve_t0<<<1, 1, 0, s->stream>>>(s->d_shared);
    SV_CU(cudaGetLastError(), "k_serve_t0 launch");
    if (s->opt.items == 3) k_serve<3><<<s->grid, kBlock, 0, s->stream>>>(P);
    else k_serve<2><<<s->grid, kBlock, 0, s->stream>>>(P);
    SV_CU(cudaGetLastError(), "persistent kernel launch");
    SV_CU(cudaEventRecord(s->ev_kernel, s->stream), "cudaEventRecord");
    s->launched = true;
    s->launches++;
    return LB_OK;
}

lb_status ensure_running(lb_server *s) {
    const unsigned long long consumed = __atomic_load_n(&s->h_ring->consumed, __ATOMIC_ACQUIRE);
    const bool pending = consumed < s->submitted;
    const bool inflight = consumed > s->acked || pending;
    if (!inflight) return LB_OK;
    if (kernel_running(s)) return LB_OK;
    // the kernel has left (idle timeout) while work is pending or in flight
    unsigned int err = 0;
    SV_CU(cudaMemcpy(&err, &s->d_shared->error, sizeof(err), cudaMemcpyDeviceToHost), "reading kernel status");
    if (err & kErrDeadline) {
        // the launch reached its time limit with work left; every query's
        // state (slots, jobs, claims) is in device memory and no CTA left in
        // the middle of a tile, so a new launch continues them
        SV_CU(cudaMemset(&s->d_shared->error, 0, sizeof(unsigned int)), "clearing kernel status");
    }
    return launch_kernel(s);
}

}  // namespace

extern "C" {

lb_status lb_server_create(lb_graph *const *graphs, int32_t ngraphs, const lb_server_options *opt, lb_server **out) {
    if (!out) return sfail(LB_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!graphs || ngraphs < 1 || ngraphs > 4096) return sfail(LB_ERR_ARG, "need 1..4096 graphs");
    lb_server *s = new (std::nothrow) lb_server();
    if (!s) return sfail(LB_ERR_OOM, "host allocation failed");
    lb_server_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.tile == 0) o.tile = 8192;
    if (o.idle_us == 0) o.idle_us = 1000;
    if (o.mem_fraction <= 0.0) o.mem_fraction = 0.5;
    if (o.launch_ms == 0) o.launch_ms = 600000;
    if (o.items == 0) o.items = 2;
    if (o.tile < 256 || o.tile > 8192 || o.tile % 256 || o.slots < 0 || o.slots > kMaxSlots || o.idle_us < 0 ||
        o.mem_fraction > 0.95 || o.ctas_per_sm < 0 || o.ctas_per_sm > 32 || o.launch_ms < 0 || o.policy < 0 ||
        o.policy > 1 || (o.items != 2 && o.items != 3)) {
        delete s;
        return sfail(LB_ERR_ARG, "bad server options");
    }
    s->opt = o;
    lb_status st = LB_OK;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    std::vector<GraphDev> gd;
    for (int32_t i = 0; i < ngraphs; ++i) {
        lb_graph *g = graphs[i];
        if (!g) { delete s; return sfail(LB_ERR_ARG, "graph handle is NULL"); }
        int64_t n = 0, m = 0;
        int32_t wgt = 0, dev = -1;
        lb_graph_info(g, &n, &m, &wgt, &dev);
        if (dev != s->device) { delete s; return sfail(LB_ERR_ARG, "every graph must live on the current device"); }
        GraphDev d;
        graph_device_arrays(g, &d.off, &d.col, &d.w);
        d.n = n;
        d.m = m;
        gd.push_back(d);
        s->graphs.push_back(g);
        s->graph_n.push_back(n);
        s->graph_m.push_back(m);
        s->graph_weighted.push_back(wgt != 0);
        if (n > s->slot_n) s->slot_n = n;
    }
    // the workspace pool: mem_fraction of free HBM, but no more than every
    // slot holding a query on the largest graph needs
    for (int32_t i = 0; i < ngraphs; ++i)
        if ((int64_t)query_bytes(s, i) > s->slot_bytes) s->slot_bytes = (int64_t)query_bytes(s, i);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->nslots = o.slots > 0 ? o.slots : 256;
    const uint64_t budget = (uint64_t)((double)free_b * o.mem_fraction) & ~(uint64_t)255u;
    const uint64_t need = (uint64_t)s->slot_bytes * (uint64_t)s->nslots;
    s->pool_bytes = budget < need ? budget : need;
    if (s->pool_bytes < (uint64_t)s->slot_bytes) {
        destroy_server(s);
        return sfail(LB_ERR_OOM, "not enough free device memory for one query on the largest graph");
    }
    int occ = 0;
    if (o.items == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve<3>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve<2>, kBlock, 0);
    if (occ < 1) occ = 1;
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < occ) occ = o.ctas_per_sm;
    s->grid = occ * s->sms;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_kernel, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_ring, sizeof(HostShared), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        memset(s->h_ring, 0, sizeof(HostShared));
        e = cudaHostGetDevicePointer((void **)&s->d_ring, s->h_ring, 0);
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->pool, (size_t)s->pool_bytes);
    if (e == cudaSuccess) {
        s->free_ranges[0] = s->pool_bytes;
        s->pool_free = s->pool_bytes;
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_graphs, sizeof(GraphDev) * gd.size());
    if (e == cudaSuccess) e = cudaMemcpy(s->d_graphs, gd.data(), sizeof(GraphDev) * gd.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_shared, sizeof(Shared));
    if (e == cudaSuccess) e = cudaMemset(s->d_shared, 0, sizeof(Shared));
    if (e == cudaSuccess) e = cudaMemset(&s->d_shared->oldest, 0xFF, sizeof(unsigned long long));  // kNoOldest
    std::vector<Slot> hs((size_t)s->nslots);
    for (Slot &S : hs) memset(&S, 0, sizeof(Slot));
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_slots, sizeof(Slot) * (size_t)s->nslots);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_slots, hs.data(), sizeof(Slot) * (size_t)s->nslots, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = sfail(e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, "server set-up", e);
        destroy_server(s);
        return st;
    }
    *out = s;
    return LB_OK;
}

lb_status lb_server_destroy(lb_server *s) {
    destroy_server(s);
    return LB_OK;
}

lb_status lb_server_info(const lb_server *s, lb_server_info_t *info) {
    if (!s || !info) return sfail(LB_ERR_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->slots = s->nslots;
    info->grid = s->grid;
    info->slot_bytes = s->slot_bytes;
    info->slot_n = s->slot_n;
    info->kernel_launches = (int64_t)s->launches;
    info->submitted = (int64_t)(s->submitted + s->pending.size());
    info->completed = (int64_t)s->acked;
    info->pool_bytes = (int64_t)s->pool_bytes;
    info->pool_free = (int64_t)s->pool_free;
    info->pending = (int64_t)s->pending.size();
    return LB_OK;
}

lb_status lb_server_submit(lb_server *s, int32_t graph, int32_t src, int32_t kind, void *out_dev, uint64_t *ticket) {
    if (!s || !out_dev) return sfail(LB_ERR_ARG, "NULL argument");
    if (graph < 0 || graph >= (int32_t)s->graphs.size()) return sfail(LB_ERR_ARG, "graph index out of range");
    if (src < 0 || (int64_t)src >= s->graph_n[(size_t)graph]) return sfail(LB_ERR_ARG, "source out of range");
    if (kind != LB_KIND_BFS && kind != LB_KIND_SSSP) return sfail(LB_ERR_ARG, "kind must be LB_KIND_BFS or LB_KIND_SSSP");
    if (kind == LB_KIND_SSSP && !s->graph_weighted[(size_t)graph]) return sfail(LB_ERR_UNSUPPORTED, "SSSP needs a weighted graph");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->submitted - s->acked + s->pending.size() >= kRing)
        return sfail(LB_ERR_UNSUPPORTED, "request ring full: poll completions first");
    const uint64_t bytes = query_bytes(s, graph);
    if (bytes > s->pool_bytes) return sfail(LB_ERR_OOM, "the query needs more device memory than the server's pool");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    lb_server::Pending q;
    q.graph = graph;
    q.src = src;
    q.kind = kind;
    q.out = (unsigned long long)(uintptr_t)out_dev;
    q.ticket = s->next_ticket++;
    q.bytes = bytes;
    if (ticket) *ticket = q.ticket;
    s->pending.push_back(q);
    pump(s);  // admitted to the device once its workspace fits in the pool
    lb_status st = ensure_running(s);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    return st;
}

lb_status lb_server_poll(lb_server *s, lb_completion *out, int32_t cap, int32_t *ndone) {
    if (!s || !ndone || (cap > 0 && !out)) return sfail(LB_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    int32_t k = 0;
    while (k < cap) {
        Done &d = s->h_ring->done[s->acked % kRing];
        const unsigned long long seq = __atomic_load_n(&d.seq, __ATOMIC_ACQUIRE);
        if (seq != s->acked + 1ull) break;
        out[k].ticket = d.ticket;
        out[k].status = d.status;
        out[k].graph = d.graph;
        out[k].iterations = d.iterations;
        out[k].edges_relaxed = (int64_t)d.edges_relaxed;
        out[k].device_ns = (int64_t)(d.t_done_ns - d.t_admit_ns);
        auto h = s->held.find(d.ticket);  // the query's workspace returns to the pool
        if (h != s->held.end()) {
            pool_release(s, h->second.first, h->second.second);
            s->held.erase(h);
        }
        ++k;
        s->acked++;
    }
    *ndone = k;
    pump(s);
    lb_status st = ensure_running(s);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    return st;
}

lb_status lb_server_state(lb_server *s, lb_server_state_t *out) {
    if (!s || !out) return sfail(LB_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    // read through a side stream: the persistent kernel may be running
    cudaStream_t side = nullptr;
    lb_status st = LB_OK;
    Shared sh;
    std::vector<Slot> slots((size_t)s->nslots);
    cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sh, s->d_shared, sizeof(Shared), cudaMemcpyDeviceToHost, side);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(slots.data(), s->d_slots, sizeof(Slot) * slots.size(), cudaMemcpyDeviceToHost, side);
    if (e == cudaSuccess) e = cudaStreamSynchronize(side);
    if (side) cudaStreamDestroy(side);
    if (e != cudaSuccess) {
        st = sfail(LB_ERR_CUDA, "reading server state", e);
    } else {
        out->submitted = (int64_t)s->submitted;
        out->consumed = (int64_t)sh.consumed;
        out->completed = (int64_t)sh.completed;
        out->acked = (int64_t)s->acked;
        out->active = (int32_t)sh.active;
        out->stopping = (int32_t)sh.stopping;
        out->admit_lock = (int32_t)sh.admit_lock;
        out->kernel_error = (int32_t)sh.error;
        out->kernel_running = kernel_running(s) ? 1 : 0;
        for (int i = 0; i < 8; ++i) out->prof[i] = (int64_t)sh.prof[i];
        int32_t k = 0;
        for (size_t i = 0; i < slots.size(); ++i) {
            const Slot &S = slots[i];
            if (!S.busy) continue;
            out->busy_slots++;
            if (k < 16) {
                lb_slot_state_t &d = out->slot[k++];
                d.slot = (int32_t)i;
                d.graph = S.graph;
                d.kind = S.kind;
                d.level = (int32_t)S.level;
                d.job_kind = (int32_t)job_kind(S.job);
                d.job_tiles = (int32_t)job_tiles(S.job);
                d.job_done = (int32_t)S.job_done;
                d.job_gen = (int32_t)job_gen(S.job);
                d.claim = (int64_t)S.claim;
                d.in_cnt = (int64_t)S.in_cnt;
                d.in_edges = (int64_t)S.in_edges;
                d.error = (int32_t)S.error;
                d.ticket = (int64_t)S.ticket;
            }
        }
        out->listed = k;
    }
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    return st;
}

lb_status lb_server_autotune(lb_graph *const *graphs, int32_t ngraphs, const lb_server_options *base,
                             const int32_t *req_graph, const int32_t *req_src, const int32_t *req_kind, int32_t nreq,
                             lb_server_options *best, double *best_qps) {
    if (!graphs || ngraphs < 1 || !req_graph || !req_src || !req_kind || nreq < 1 || nreq > 4096)
        return sfail(LB_ERR_ARG, "need graphs and 1..4096 sample requests");
    for (int32_t i = 0; i < nreq; ++i) {
        if (req_graph[i] < 0 || req_graph[i] >= ngraphs || !graphs[req_graph[i]]) return sfail(LB_ERR_ARG, "bad request graph");
        int64_t n = 0, m = 0;
        int32_t w = 0, dev = 0;
        lb_graph_info(graphs[req_graph[i]], &n, &m, &w, &dev);
        if (req_src[i] < 0 || (int64_t)req_src[i] >= n) return sfail(LB_ERR_ARG, "bad request source");
        if (req_kind[i] != LB_KIND_BFS && (req_kind[i] != LB_KIND_SSSP || !w)) return sfail(LB_ERR_ARG, "bad request kind");
    }
    lb_server_options o0;
    memset(&o0, 0, sizeof(o0));
    if (base) o0 = *base;
    // one output buffer per sample request, sized for its graph
    std::vector<void *> outs((size_t)nreq, nullptr);
    lb_status st = LB_OK;
    for (int32_t i = 0; i < nreq && st == LB_OK; ++i) {
        int64_t n = 0;
        lb_graph_info(graphs[req_graph[i]], &n, nullptr, nullptr, nullptr);
        if (cudaMalloc(&outs[(size_t)i], 4 * (size_t)n) != cudaSuccess) st = sfail(LB_ERR_OOM, "sample output buffers");
    }
    double top = -1.0;
    lb_server_options top_o = o0;
    std::vector<lb_completion> done(256);
    // candidate grid: edges per lane, CTAs per SM, largest tile, claiming policy
    for (int32_t items : {2, 3})
        for (int32_t ctas : {0, 3})
            for (int32_t tile : {4096, 8192})
                for (int32_t policy : {0, 1}) {
                    if (st != LB_OK) break;
                    lb_server_options o = o0;
                    o.items = items;
                    o.ctas_per_sm = ctas;
                    o.tile = tile;
                    o.policy = policy;
                    lb_server *s = nullptr;
                    st = lb_server_create(graphs, ngraphs, &o, &s);
                    if (st != LB_OK) break;
                    double dt = 0.0;
                    for (int rep = 0; rep < 2 && st == LB_OK; ++rep) {  // the first run warms up
                        const auto t0 = std::chrono::steady_clock::now();
                        for (int32_t i = 0; i < nreq && st == LB_OK; ++i)
                            st = lb_server_submit(s, req_graph[i], req_src[i], req_kind[i], outs[(size_t)i], nullptr);
                        int32_t left = nreq;
                        while (left > 0 && st == LB_OK) {
                            int32_t nd = 0;
                            st = lb_server_poll(s, done.data(), (int32_t)done.size(), &nd);
                            left -= nd;
                            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(300))
                                st = sfail(LB_ERR_TIMEOUT, "a sample batch ran past 300 s");
                        }
                        dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                    }
                    lb_server_destroy(s);
                    if (st == LB_OK && nreq / dt > top) {
                        top = nreq / dt;
                        top_o = o;
                    }
                }
    for (void *p : outs)
        if (p) cudaFree(p);
    if (st != LB_OK) return st;
    if (best) *best = top_o;
    if (best_qps) *best_qps = top;
    return LB_OK;
}

lb_status lb_server_stop(lb_server *s) {
    if (!s) return sfail(LB_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    __atomic_store_n(&s->h_ring->stop, 1u, __ATOMIC_RELEASE);
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->launched = false;
    __atomic_store_n(&s->h_ring->stop, 0u, __ATOMIC_RELEASE);
    return LB_OK;
}

}  // extern "C"
