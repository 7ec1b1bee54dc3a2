// Device building blocks shared by the step kernels of every strategy.
//
//  * Relax ops (the relaxation of the paper's EP and WD algorithms: a
//    destination whose distance exceeds the source's distance plus the
//    edge weight takes that sum and is pushed):
//      BFS  - claim v with atomicOr on a visited bitmap, level[v] = L + 1;
//      SSSP - atomicMin on dist[v]; queue v only for the first improvement
//             in an iteration (atomicOr on the iteration's queued bitmap),
//             so a list never exceeds n.
//    Both run test-then-atomic: the plain read can only be stale in the
//    direction that costs an extra atomic, never one that loses an update.
//    In the WD kernels the atomics are deferred: the relax buffers the
//    candidates that pass the plain test, and the flush makes the atomics
//    of a whole buffer at once (FlushOut::defer).
//  * Warp push buffers: the paper pushes with one atomic per node ("work
//    chunking", Sec. II-B / IV-D).  Here a warp collects up to kWB pushed
//    nodes in shared memory and reserves their list slots and their edges
//    with ONE 64-bit atomicAdd on a packed (entries << 32 | edges) counter.
//    The reservation returns consistent bases for both, so each entry's
//    edge prefix (the WD prefix sum of Sec. III-A, Thrust's inclusive scan
//    in the paper) and the WD tile starts (the paper's find_offsets) come
//    out of the push itself: no scan or offset kernel runs per iteration.
//  * The last CTA of every step kernel finalises the iteration (swaps the
//    lists, records the trace, sets the CUDA-graph loop condition), so each
//    iteration is a single kernel launch.
#pragma once

#include "lb_internal.cuh"

namespace lbk {

// Entries per warp push buffer (a multiple of 32).  192 measured 23% slower
// (BFS) at R-MAT scale 24: the larger shared-memory footprint costs
// resident CTAs.
#ifndef LB_KWB
#define LB_KWB 128
#endif
constexpr int kWB = LB_KWB;
constexpr unsigned kFull = 0xFFFFFFFFu;

// what a flush writes
enum : int { kOutNode = 0, kOutGranule = 1, kOutEdges = 2, kOutEdgesPerEdge = 3, kOutPhys = 4 };

// A warp's push buffer of N entries in shared memory.  The shared-memory
// footprint sets the L1 / shared-memory carve-out: a smaller buffer leaves
// more L1 for the randomly read visited bitmap (BFS).
template <int N>
struct WarpBufT {
    static constexpr int kCap = N;
    int32_t beg[N];
    int32_t v[N];
    uint32_t deg[N];
};
using WarpBuf = WarpBufT<kWB>;

// Prefix scratch of a flush that expands entries into granules or edges (a
// binary search over the output units); node flushes need none.
template <int N>
struct WarpScratchT {
    uint32_t pu[N];  // exclusive prefix of output units
    uint32_t pe[N];  // exclusive prefix of edges
};
using WarpScratch = WarpScratchT<kWB>;
struct NoScratch {};

struct FlushOut {
    NodeList list;     // node / granule output
    int32_t *elist;    // edge-id output
    unsigned long long *pack;
    uint32_t *err;               // error word (capacity overflow)
    unsigned long long *pushes;  // push counter
    const int32_t *child_first;  // kOutPhys: first child id of each split node
    int64_t cap;       // entries the output can hold
    int64_t tile_cap;  // tstart entries
    int32_t tile;      // edges between recorded tile starts (kTileGrain in the hot path)
    int32_t mdt;
    // deferred offsets (kOutNode): the pushes buffered only the vertex, and
    // the flush loads every buffered vertex's first edge and degree from
    // `off` (all entries at once, so one latency per flush instead of one per
    // relax group) and drops vertices without out-edges
    const int64_t *off = nullptr;
    int32_t defer = 0;
    // defer == 3 (SSSP): the buffer holds (vertex, offered distance) pairs
    // whose plain check passed; the flush makes their atomicMin and, for
    // the improved vertices, the queued-bit claim.
    // defer == 2 (BFS): the buffer holds visited-check candidates, not yet
    // claimed; the flush claims them all at once (one atomicOr per entry,
    // every claim of the warp in flight together), writes the new level of
    // the vertices it won and drops the rest with the vertices that have no
    // out-edges.  The claim then leaves each relax group's chain of
    // dependent accesses.
    uint32_t *claim_bitmap = nullptr;
    uint32_t *claim_status = nullptr;
    uint32_t claim_level = 0;
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <int KIND>
__device__ __forceinline__ uint32_t out_units(uint32_t deg, int32_t mdt) {
    if (KIND == kOutEdges) return deg;
    if (KIND == kOutGranule || KIND == kOutPhys)
        return deg <= (uint32_t)mdt ? 1u : (deg + (uint32_t)mdt - 1u) / (uint32_t)mdt;
    return 1u;
}

// Warp-uniform: every lane of the warp calls it with the same cnt.
// Requires cnt + 32 <= capacity on entry.  The warp synchronises its buffer
// writes here (LB_PUSH_SYNC = 1) or once at the start of the flush that
// reads them (0).
#ifndef LB_PUSH_SYNC
#define LB_PUSH_SYNC 1
#endif
template <class WB>
__device__ __forceinline__ void wpush(WB &b, uint32_t &cnt, bool want, int32_t v, int64_t beg, uint32_t deg) {
    // beg < m < 2^31: stored in 32 bits
    const unsigned m = __ballot_sync(kFull, want);
    if (want) {
        const uint32_t s = cnt + __popc(m & lanemask_lt());
        b.v[s] = v;
        b.beg[s] = (int32_t)beg;
        b.deg[s] = deg;
    }
    cnt += __popc(m);
    if (LB_PUSH_SYNC) __syncwarp();
}

// largest i in [0, n) with a[i] <= x (a[0] <= x assumed)
__device__ __forceinline__ uint32_t smem_upper(const uint32_t *a, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Warp-uniform flush of a warp push buffer into a global list.  It runs
// once per ~100 pushes; LB_FLUSH_NOINLINE=1 keeps it out of line so its
// registers do not count against the relax loops around it.
#ifndef LB_FLUSH_NOINLINE
#define LB_FLUSH_NOINLINE 0
#endif
#if LB_FLUSH_NOINLINE
#define LB_FLUSH_INLINE __noinline__
#else
#define LB_FLUSH_INLINE inline
#endif

// Output units of buffered entry i (a node list entry; with deferred
// offsets 0 for a node without out-edges, which is dropped).
template <int KIND, class WB>
__device__ __forceinline__ uint32_t entry_units(const WB &b, uint32_t i, uint32_t cnt, const FlushOut &o,
                                                uint32_t &d) {
    d = i < cnt ? b.deg[i] : 0u;
    return (i < cnt && !(KIND == kOutNode && o.defer && d == 0u)) ? out_units<KIND>(d, o.mdt) : 0u;
}

// Inclusive warp scan of (u, e) pairs.
__device__ __forceinline__ void warp_scan2(uint32_t &iu, uint32_t &ie, uint32_t lane) {
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const uint32_t tu = __shfl_up_sync(kFull, iu, k);
        const uint32_t te = __shfl_up_sync(kFull, ie, k);
        if ((int)lane >= k) { iu += tu; ie += te; }
    }
}

// The two halves of a flush.  The first completes the buffered entries
// (deferred claims and offsets) and totals their output units and edges;
// for granule / edge outputs it also stores each entry's exclusive prefix
// in `s` for the expansion.  The second writes the entries at the list
// position / edge prefix `old` (packed entries << 32 | edges) reserved for
// them; a node flush recomputes its prefix there with a warp scan per 32
// entries, so it needs no scratch.
template <int KIND, class WB, class WS>
__device__ __forceinline__ void wflush_prefix(WB &b, WS &s, uint32_t cnt, const FlushOut &o, uint32_t &run_u,
                                              uint32_t &run_e) {
    const uint32_t lane = lane_id();
    run_u = 0;
    run_e = 0;
    if (KIND == kOutNode && o.defer == 2) {
        constexpr int kPer = WB::kCap / 32;
        int32_t cv[kPer];
        uint32_t pv[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = lane + 32u * k;
            cv[k] = i < cnt ? b.v[i] : -1;
            pv[k] = 0xFFFFFFFFu;
            if (cv[k] >= 0) pv[k] = atomicOr(o.claim_bitmap + ((uint32_t)cv[k] >> 5), 1u << ((uint32_t)cv[k] & 31u));
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = lane + 32u * k;
            const bool won = cv[k] >= 0 && !((pv[k] >> ((uint32_t)cv[k] & 31u)) & 1u);
            int32_t b0 = 0, d = 0;
            if (won) {
                o.claim_status[cv[k]] = o.claim_level + 1u;
                // offsets are < m < 2^31 (checked when the graph is created)
                b0 = (int32_t)__ldg(o.off + cv[k]);
                d = (int32_t)__ldg(o.off + cv[k] + 1) - b0;
            }
            if (i < cnt) {
                b.beg[i] = b0;
                b.deg[i] = (uint32_t)d;
            }
        }
        __syncwarp();
    } else if (KIND == kOutNode && o.defer == 3) {
        // SSSP: entry i holds a candidate vertex and the distance it was
        // offered (in beg); the atomicMin of every entry, then the queued
        // bit of every improved vertex, all in flight together
        constexpr int kPer = WB::kCap / 32;
        int32_t cv[kPer];
        uint32_t pv[kPer], val[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = lane + 32u * k;
            cv[k] = i < cnt ? b.v[i] : -1;
            val[k] = i < cnt ? (uint32_t)b.beg[i] : 0u;
            pv[k] = 0u;
            if (cv[k] >= 0) pv[k] = atomicMin(o.claim_status + cv[k], val[k]);
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const bool improved = cv[k] >= 0 && val[k] < pv[k];
            if (improved && val[k] == kSat) atomicOr(o.err, kErrSaturated);
            pv[k] = 0xFFFFFFFFu;
            if (improved)
                pv[k] = atomicOr(o.claim_bitmap + ((uint32_t)cv[k] >> 5), 1u << ((uint32_t)cv[k] & 31u));
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = lane + 32u * k;
            // queued by the first improvement of this iteration only
            const bool first = cv[k] >= 0 && !((pv[k] >> ((uint32_t)cv[k] & 31u)) & 1u);
            int32_t b0 = 0, d = 0;
            if (first) {
                // offsets are < m < 2^31 (checked when the graph is created)
                b0 = (int32_t)__ldg(o.off + cv[k]);
                d = (int32_t)__ldg(o.off + cv[k] + 1) - b0;
            }
            if (i < cnt) {
                b.beg[i] = b0;
                b.deg[i] = (uint32_t)d;
            }
        }
        __syncwarp();
    } else if (KIND == kOutNode && o.defer) {
        // offsets are < m < 2^31 (checked when the graph is created)
        for (uint32_t i = lane; i < cnt; i += 32) {
            const int32_t v = b.v[i];
            const int32_t b0 = (int32_t)__ldg(o.off + v);
            b.beg[i] = b0;
            b.deg[i] = (uint32_t)((int32_t)__ldg(o.off + v + 1) - b0);
        }
        __syncwarp();
    }
    if constexpr (KIND == kOutNode) {
        uint32_t su = 0, se = 0;
        for (uint32_t i = lane; i < cnt; i += 32) {
            uint32_t d;
            su += entry_units<KIND>(b, i, cnt, o, d);
            se += d;
        }
        run_u = __reduce_add_sync(kFull, su);
        run_e = __reduce_add_sync(kFull, se);
    } else {
        for (uint32_t c = 0; c < cnt; c += 32) {
            const uint32_t i = c + lane;
            uint32_t d;
            const uint32_t u = entry_units<KIND>(b, i, cnt, o, d);
            uint32_t iu = u, ie = d;
            warp_scan2(iu, ie, lane);
            if (i < cnt) { s.pu[i] = run_u + iu - u; s.pe[i] = run_e + ie - d; }
            run_u += __shfl_sync(kFull, iu, 31);
            run_e += __shfl_sync(kFull, ie, 31);
        }
    }
}

template <int KIND, bool TILED, class WB, class WS>
__device__ __forceinline__ void wflush_write(const WB &b, const WS &s, uint32_t &cnt, const FlushOut &o,
                                             unsigned long long old, uint32_t run_u) {
    const uint32_t lane = lane_id();
    const int64_t ubase = (int64_t)(old >> 32);
    const int64_t ebase = (int64_t)(old & 0xFFFFFFFFull);
    if (ubase + (int64_t)run_u > o.cap) {
        if (lane == 0) atomicOr(o.err, kErrCapacity);
        cnt = 0;
        __syncwarp();
        return;
    }
    if constexpr (KIND == kOutNode) {
        uint32_t ru = 0, re = 0;
        for (uint32_t c = 0; c < cnt; c += 32) {
            const uint32_t i = c + lane;
            uint32_t d;
            const uint32_t u = entry_units<KIND>(b, i, cnt, o, d);
            uint32_t iu = u, ie = d;
            warp_scan2(iu, ie, lane);
            if (u) {  // a node list entry (deferred offsets: one with out-edges)
                const int64_t pos = ubase + ru + iu - u;
                const int64_t S = ebase + re + ie - d;
                o.list.v[pos] = b.v[i];
                o.list.beg[pos] = b.beg[i];
                o.list.scan[pos] = (int32_t)S;
                if (TILED) {
                    const int64_t E = S + d;
                    if (o.tile == (int32_t)kTileGrain) {  // the hot path: shifts, no division
                        for (int64_t k = (S + kTileGrain - 1) >> 8; (k << 8) < E; ++k)
                            if (k < o.tile_cap) o.list.tstart[k] = (int32_t)pos;
                    } else {
                        for (int64_t k = (S + o.tile - 1) / o.tile; k * o.tile < E; ++k)
                            if (k < o.tile_cap) o.list.tstart[k] = (int32_t)pos;
                    }
                }
            }
            ru += __shfl_sync(kFull, iu, 31);
            re += __shfl_sync(kFull, ie, 31);
        }
    } else {
        for (uint32_t j = lane; j < run_u; j += 32) {
            const uint32_t i = smem_upper(s.pu, cnt, j);
            const int64_t k = (int64_t)(j - s.pu[i]);
            if (KIND == kOutGranule || KIND == kOutPhys) {
                const int64_t pos = ubase + j;
                // a physically split node's runs after the first belong to its children
                o.list.v[pos] = (KIND == kOutPhys && k > 0) ? __ldg(o.child_first + b.v[i]) + (int32_t)(k - 1) : b.v[i];
                o.list.beg[pos] = (int32_t)(b.beg[i] + k * o.mdt);
                o.list.scan[pos] = (int32_t)(ebase + s.pe[i] + k * o.mdt);
            } else {
                o.elist[ubase + j] = (int32_t)(b.beg[i] + k);
            }
        }
    }
    cnt = 0;
    __syncwarp();
}

template <int KIND, bool TILED, class WB, class WS>
__device__ LB_FLUSH_INLINE void wflush(WB &b, WS &s, uint32_t &cnt, const FlushOut &o) {
    if (cnt == 0) return;
    if (!LB_PUSH_SYNC) __syncwarp();
    const uint32_t lane = lane_id();
    uint32_t run_u, run_e;
    wflush_prefix<KIND>(b, s, cnt, o, run_u, run_e);
    unsigned long long old = 0;
    if (lane == 0) {
        old = atomicAdd(o.pack, ((unsigned long long)run_u << 32) | (unsigned long long)run_e);
        atomicAdd(o.pushes, (unsigned long long)run_u);
    }
    old = __shfl_sync(kFull, old, 0);
    __syncwarp();
    wflush_write<KIND, TILED>(b, s, cnt, o, old, run_u);
}

// Block-wide flush of every warp's buffer (every thread of the block calls
// it): one list reservation per CTA instead of one per warp.  At the end of
// an iteration every warp with pushes flushes at once, and on lists with
// many small pushes (a grid's SSSP wavefront) thousands of same-address
// atomics per iteration would queue at one L2 slice.  The packed add is
// exact: a list's entries and its edges (< m < 2^31) each fit their half.
template <int KIND, bool TILED, class WB, class WS>
__device__ void wflush_block(WB &b, WS &s, uint32_t &cnt, const FlushOut &o) {
    __shared__ unsigned long long s_tot[kWarps];
    __shared__ unsigned long long s_base;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    __syncwarp();
    uint32_t run_u = 0, run_e = 0;
    if (cnt) wflush_prefix<KIND>(b, s, cnt, o, run_u, run_e);
    if (lane == 0) s_tot[warp] = ((unsigned long long)run_u << 32) | (unsigned long long)run_e;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int w = 0; w < kWarps; ++w) {
            const unsigned long long t = s_tot[w];
            s_tot[w] = sum;
            sum += t;
        }
        s_base = sum ? atomicAdd(o.pack, sum) : 0ull;
        if (sum) atomicAdd(o.pushes, sum >> 32);
    }
    __syncthreads();
    if (cnt) wflush_write<KIND, TILED>(b, s, cnt, o, s_base + s_tot[warp], run_u);
    cnt = 0;
}

// ---- relax ops ------------------------------------------------------------

// BFS: true iff this thread discovered v (and set its level).
__device__ __forceinline__ bool bfs_claim(uint32_t *__restrict__ bitmap, uint32_t *__restrict__ status, int32_t v,
                                          uint32_t newlev) {
    const uint32_t word = (uint32_t)v >> 5, bit = 1u << ((uint32_t)v & 31u);
    if (bitmap[word] & bit) return false;
    if (atomicOr(&bitmap[word], bit) & bit) return false;
    status[v] = newlev;
    return true;
}

// SSSP queued bits.  Iteration L sets the bit of every vertex it queues in
// half (L & 1) of the bitmap and clears half ((L + 1) & 1), which no one
// reads during iteration L, for iteration L + 1.  (A per-vertex stamp of
// the queueing iteration would carry the same information in 32x the
// bytes; these bits stay in L2 beside the distances.)
__device__ __forceinline__ uint32_t *queued_half(uint32_t *bitmap, int64_t words, uint32_t level) {
    return bitmap + (level & 1u) * words;
}

template <bool COH>
__device__ __forceinline__ bool is_queued(const uint32_t *q, int32_t u) {
    const uint32_t x = COH ? __ldcg(q + ((uint32_t)u >> 5)) : q[(uint32_t)u >> 5];
    return (x >> ((uint32_t)u & 31u)) & 1u;
}

// Clears the other half of the queued bitmap with the whole grid: 16-byte
// stores (words is a multiple of 4) when the half is 16-byte aligned, as
// every allocation from cudaMalloc is; 4-byte stores otherwise.
__device__ __forceinline__ void clear_next_queued(uint32_t *bitmap, int64_t words, uint32_t level) {
    uint32_t *h = queued_half(bitmap, words, level + 1u);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((uintptr_t)h & 15u) == 0) {
        uint4 *q = reinterpret_cast<uint4 *>(h);
        for (int64_t i = tid; i < words / 4; i += stride) q[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (int64_t i = tid; i < words; i += stride) h[i] = 0u;
    }
}

// SSSP: true iff v improved and this is v's first queueing this iteration.
__device__ __forceinline__ bool sssp_relax(uint32_t *__restrict__ status, uint32_t *__restrict__ q, int32_t v,
                                           uint32_t du, uint32_t w, Ctl *ctl) {
    if (du == kInf) return false;
    const uint64_t a64 = (uint64_t)du + (uint64_t)w;
    const uint32_t alt = a64 >= kSat ? kSat : (uint32_t)a64;
    if (alt >= status[v]) return false;
    const uint32_t old = atomicMin(&status[v], alt);
    if (alt >= old) return false;
    if (alt == kSat) atomicOr(&ctl->error, kErrSaturated);
    if (is_queued<false>(q, v)) return false;
    const uint32_t bit = 1u << ((uint32_t)v & 31u);
    return !(atomicOr(&q[(uint32_t)v >> 5], bit) & bit);
}

// SSSP: distance a worklist entry u relaxes with.  When u has already been
// queued again in this iteration (its bit is set), its distance improved
// after it was listed and the next iteration expands it with that newer
// value, so expanding it now is redundant work: return kInf, which makes
// every relaxation from u a no-op.
__device__ __forceinline__ uint32_t sssp_source_dist(const uint32_t *__restrict__ status, const uint32_t *q,
                                                     int32_t u) {
    return is_queued<false>(q, u) ? kInf : status[u];
}

// Relaxes ITEMS loaded edges of a warp and pushes the vertices that must be
// queued.  The relax runs in stages over all items -- plain checks, then
// every atomic, then every offset load of a won vertex, then the pushes --
// so the latencies of the items overlap instead of queueing behind one
// another (a warp-synchronous push between items would serialise them).
// Loads of data other CTAs write: plain (L1) inside a single-iteration
// launch, L2-coherent (ld.global.cg) inside the persistent serving kernel.
// BFS visited check through L2 (1) instead of L1 (0): sees other SMs'
// claims sooner at the cost of L2 latency (measured 31% slower at R-MAT
// scale 24).
#ifndef LB_BFS_BITMAP_CG
#define LB_BFS_BITMAP_CG 0
#endif
template <bool COH>
__device__ __forceinline__ uint32_t ld_mut(const uint32_t *p) {
    return COH ? __ldcg(p) : *p;
}

// Warp-uniform early exits in relax_items: after the checks when no lane
// has a candidate, after the atomics when no lane won one.  Measured on
// R-MAT scale 24: SSSP 8.98 -> 8.53 ms per query.
#ifndef LB_EARLY_EXIT
#define LB_EARLY_EXIT 1
#endif
// FLUSH = false: the caller flushes; then cnt + 32 * ITEMS <= capacity on entry.
// With FlushOut::defer set (kOutNode) only the vertex is buffered.
template <bool SSSP, int ITEMS, int KIND, bool TILED, bool COH = false, bool FLUSH = true, class WB, class WS>
__device__ __forceinline__ void relax_items(const bool (&ok)[ITEMS], const int32_t (&vv)[ITEMS],
                                            const uint32_t (&ww)[ITEMS], const uint32_t (&dd)[ITEMS],
                                            const int64_t *__restrict__ off, uint32_t *__restrict__ bitmap,
                                            uint32_t *__restrict__ qcur, uint32_t *__restrict__ status,
                                            uint32_t level, uint32_t *err, WB &wb,
                                            WS &ws, uint32_t &cnt, const FlushOut &o) {
    bool cand[ITEMS];
    uint32_t val[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        cand[it] = false;
        val[it] = 0;
        if (!ok[it]) continue;
        if (SSSP) {
            if (dd[it] == kInf) continue;
            // dd + w saturated at kSat: a 32-bit sum that wrapped (s < dd) or
            // reached kSat is exactly the case of the 64-bit sum >= kSat
            const uint32_t s32 = dd[it] + ww[it];
            val[it] = (s32 < dd[it] || s32 >= kSat) ? kSat : s32;
            cand[it] = val[it] < ld_mut<COH>(status + vv[it]);
        } else {
            cand[it] = !(ld_mut<COH || LB_BFS_BITMAP_CG>(bitmap + ((uint32_t)vv[it] >> 5)) & (1u << ((uint32_t)vv[it] & 31u)));
        }
    }
    if (LB_EARLY_EXIT) {
        bool any = false;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) any = any || cand[it];
        if (!__any_sync(kFull, any)) return;
    }
    uint32_t prev[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        prev[it] = 0;
        if (!cand[it]) continue;
        if (SSSP) prev[it] = atomicMin(&status[vv[it]], val[it]);
        else prev[it] = atomicOr(&bitmap[(uint32_t)vv[it] >> 5], 1u << ((uint32_t)vv[it] & 31u));
    }
    bool won[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        if (SSSP) {
            won[it] = cand[it] && val[it] < prev[it];
            if (won[it] && val[it] == kSat) atomicOr(err, kErrSaturated);
        } else {
            won[it] = cand[it] && !(prev[it] & (1u << ((uint32_t)vv[it] & 31u)));
            if (won[it]) status[vv[it]] = level + 1;
        }
    }
    if (SSSP) {
        // queue only the first improvement of v in this iteration
#pragma unroll
        for (int it = 0; it < ITEMS; ++it)
            if (won[it] && is_queued<COH>(qcur, vv[it])) won[it] = false;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it)
            if (won[it]) prev[it] = atomicOr(&qcur[(uint32_t)vv[it] >> 5], 1u << ((uint32_t)vv[it] & 31u));
#pragma unroll
        for (int it = 0; it < ITEMS; ++it)
            if (won[it] && (prev[it] & (1u << ((uint32_t)vv[it] & 31u)))) won[it] = false;
    }
    if (LB_EARLY_EXIT) {
        bool any = false;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) any = any || won[it];
        if (!__any_sync(kFull, any)) return;
    }
    if (KIND == kOutNode && o.defer) {
        // deferred offsets: buffer the vertex only (the flush loads its offsets)
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            wpush(wb, cnt, won[it], vv[it], 0, 0u);
            if (FLUSH && cnt > WB::kCap - 32) wflush<KIND, TILED>(wb, ws, cnt, o);
        }
        return;
    }
    // offsets are < m < 2^31 (checked when the graph is created)
    int32_t vb[ITEMS], ve[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        vb[it] = 0;
        ve[it] = 0;
        if (won[it]) {
            vb[it] = (int32_t)__ldg(off + vv[it]);
            ve[it] = (int32_t)__ldg(off + vv[it] + 1);
        }
    }
    if (KIND == kOutEdgesPerEdge) {
        // no work chunking: one reservation per pushed edge id
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            if (!won[it]) continue;
            for (int64_t e = vb[it]; e < ve[it]; ++e) {
                const unsigned long long pos = atomicAdd(o.pack, (1ull << 32) | 1ull) >> 32;
                if ((int64_t)pos < o.cap) o.elist[pos] = (int32_t)e;
                else atomicOr(o.err, kErrCapacity);
            }
            atomicAdd(o.pushes, (unsigned long long)(ve[it] - vb[it]));
        }
        return;
    }
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const bool want = won[it] && ve[it] > vb[it];
        wpush(wb, cnt, want, vv[it], vb[it], (uint32_t)(ve[it] - vb[it]));
        if (FLUSH && cnt > WB::kCap - 32) wflush<KIND, TILED>(wb, ws, cnt, o);
    }
}

#ifndef LB_LEAN_PUSH_SIMPLE
#define LB_LEAN_PUSH_SIMPLE 0
#endif
// Pushes of the WD walk buffer only the vertex; the flush loads the offsets
// (FlushOut::defer).  Measured on R-MAT scale 24: BFS 2.10 -> 1.92 ms, SSSP
// 9.35 -> 9.01 ms per query (the offset loads leave each relax group's chain
// of dependent memory accesses, and the walk needs fewer registers).
#ifndef LB_DEFER_OFFSETS
#define LB_DEFER_OFFSETS 1
#endif
// BFS relax of R loaded edges per lane with warp-uniform early exits: the
// visited check for every item, then (only if some lane of the warp found
// an unvisited vertex) the claims, then (only if some lane won one) the
// level writes, offset loads and one push of all won vertices with edges.
// The push buffer is flushed only when this group's pushes would not fit,
// so flushes carry close to a full buffer.  Requires R * 32 <= capacity.
template <int R, bool COH, class WB, class WS>
__device__ __forceinline__ void relax_bfs_lean(const bool (&ok)[R], const int32_t (&vv)[R],
                                               const int64_t *__restrict__ off, uint32_t *__restrict__ bitmap,
                                               uint32_t *__restrict__ status, uint32_t level, WB &wb,
                                               WS &ws, uint32_t &cnt, const FlushOut &o) {
    static_assert(R * 32 <= WB::kCap, "push buffer too small for one group");
    uint32_t cand = 0;  // bit r: item r found v unvisited
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t x = ok[r] ? ld_mut<COH || LB_BFS_BITMAP_CG>(bitmap + ((uint32_t)vv[r] >> 5)) : 0xFFFFFFFFu;
        if (!((x >> ((uint32_t)vv[r] & 31u)) & 1u)) cand |= 1u << r;
    }
    if (!__any_sync(kFull, cand != 0u)) return;
    if (o.defer == 2) {
        // deferred claims: buffer the candidates; the flush claims them
        unsigned bal[R];
        uint32_t tot = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            bal[r] = __ballot_sync(kFull, (cand >> r) & 1u);
            tot += __popc(bal[r]);
        }
        if (cnt + tot > (uint32_t)WB::kCap) wflush<kOutNode, true>(wb, ws, cnt, o);
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((bal[r] >> lane_id()) & 1u) wb.v[cnt + __popc(bal[r] & lt)] = vv[r];
            cnt += __popc(bal[r]);
        }
        __syncwarp();
        return;
    }
    uint32_t won = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if ((cand >> r) & 1u) {
            const uint32_t bit = 1u << ((uint32_t)vv[r] & 31u);
            if (!(atomicOr(bitmap + ((uint32_t)vv[r] >> 5), bit) & bit)) won |= 1u << r;
        }
    }
    if (!__any_sync(kFull, won != 0u)) return;
    if (o.defer) {
        // level writes, then every won vertex is buffered; the flush loads
        // the offsets and drops vertices without out-edges
        unsigned bal[R];
        uint32_t tot = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((won >> r) & 1u) status[vv[r]] = level + 1;
            bal[r] = __ballot_sync(kFull, (won >> r) & 1u);
            tot += __popc(bal[r]);
        }
        if (cnt + tot > (uint32_t)WB::kCap) wflush<kOutNode, true>(wb, ws, cnt, o);
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((bal[r] >> lane_id()) & 1u) wb.v[cnt + __popc(bal[r] & lt)] = vv[r];
            cnt += __popc(bal[r]);
        }
        __syncwarp();
        return;
    }
    int32_t vb[R], vd[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        vb[r] = 0;
        vd[r] = 0;
        if ((won >> r) & 1u) {
            status[vv[r]] = level + 1;
            // offsets are < m < 2^31 (checked when the graph is created)
            vb[r] = (int32_t)__ldg(off + vv[r]);
            vd[r] = (int32_t)__ldg(off + vv[r] + 1) - vb[r];
        }
    }
#if LB_LEAN_PUSH_SIMPLE
    // flush whenever a full group might not fit, then push item by item
    if (cnt > (uint32_t)(WB::kCap - 32 * R)) wflush<kOutNode, true>(wb, ws, cnt, o);
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const unsigned b = __ballot_sync(kFull, ((won >> r) & 1u) && vd[r] > 0);
        if ((b >> lane_id()) & 1u) {
            const uint32_t s = cnt + __popc(b & lt);
            wb.v[s] = vv[r];
            wb.beg[s] = vb[r];
            wb.deg[s] = (uint32_t)vd[r];
        }
        cnt += __popc(b);
    }
#else
    unsigned bal[R];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        bal[r] = __ballot_sync(kFull, ((won >> r) & 1u) && vd[r] > 0);
        tot += __popc(bal[r]);
    }
    if (tot == 0) return;
    if (cnt + tot > (uint32_t)WB::kCap) wflush<kOutNode, true>(wb, ws, cnt, o);
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if ((bal[r] >> lane_id()) & 1u) {
            const uint32_t s = cnt + __popc(bal[r] & lt);
            wb.v[s] = vv[r];
            wb.beg[s] = vb[r];
            wb.deg[s] = (uint32_t)vd[r];
        }
        cnt += __popc(bal[r]);
    }
#endif
    __syncwarp();
}

// SSSP distance checks of the deferred relax through L2 (1) or L1 (0): the
// distance array is read at random and L1 hits are rare (11-14% at R-MAT
// scale 22).  Measured on R-MAT scale 24: with 3 edges per lane at 5 CTAs
// per SM 1.6-1.7% faster through L2; with 4 edges per lane at 4 CTAs per
// SM (the WD step now) 1.7% faster through L1 (6.59 -> 6.48 ms).
#ifndef LB_SSSP_STATUS_CG
#define LB_SSSP_STATUS_CG 0
#endif
// SSSP relax of R loaded edges per lane with deferred atomics
// (FlushOut::defer == 3): the plain distance check for every item, then
// (only if some lane found an improvement) every candidate vertex and the
// distance it offers go into the push buffer.  The flush makes the
// atomicMin and queued-bit claims of a whole buffer at once.
template <int R, bool COH, class WB, class WS>
__device__ __forceinline__ void relax_sssp_defer(const bool (&ok)[R], const int32_t (&vv)[R],
                                                 const uint32_t (&ww)[R], const uint32_t (&dd)[R],
                                                 const uint32_t *__restrict__ status, WB &wb, WS &ws,
                                                 uint32_t &cnt, const FlushOut &o) {
    static_assert(R * 32 <= WB::kCap, "push buffer too small for one group");
    uint32_t cand = 0;
    uint32_t val[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        val[r] = 0u;
        if (!ok[r] || dd[r] == kInf) continue;
        // dd + w saturated at kSat: a 32-bit sum that wrapped (s < dd) or
        // reached kSat is exactly the case of the 64-bit sum >= kSat
        const uint32_t s32 = dd[r] + ww[r];
        val[r] = (s32 < dd[r] || s32 >= kSat) ? kSat : s32;
        if (val[r] < ld_mut<COH || LB_SSSP_STATUS_CG>(status + vv[r])) cand |= 1u << r;
    }
    if (!__any_sync(kFull, cand != 0u)) return;
    unsigned bal[R];
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        bal[r] = __ballot_sync(kFull, (cand >> r) & 1u);
        tot += __popc(bal[r]);
    }
    if (cnt + tot > (uint32_t)WB::kCap) wflush<kOutNode, true>(wb, ws, cnt, o);
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if ((bal[r] >> lane_id()) & 1u) {
            const uint32_t sl = cnt + __popc(bal[r] & lt);
            wb.v[sl] = vv[r];
            wb.beg[sl] = (int32_t)val[r];
        }
        cnt += __popc(bal[r]);
    }
    __syncwarp();
}

// ---- end-of-step protocol ----------------------------------------------------

__device__ __forceinline__ bool block_is_last(Ctl *ctl) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->blocks_done, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    return s_last != 0;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}



__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void trace_append(Ctl *ctl, int32_t mode, int64_t list_size, int64_t edges) {
    const uint32_t t = ctl->trace_len;
    if (t < (uint32_t)kTraceMax) {
        ctl->trace[t].level = (int32_t)ctl->level;
        ctl->trace[t].mode = mode;
        ctl->trace[t].list_size = list_size;
        ctl->trace[t].edges = edges;
        ctl->trace[t].t_ns = (int64_t)(global_ns() - ctl->t_start);
        ctl->trace_len = t + 1;
    }
}

__device__ __forceinline__ void set_loop(const StepParams &p, Ctl *ctl, bool more) {
    if (ctl->level >= ctl->max_levels || ctl->step >= ctl->max_steps) {
        if (more) ctl->error |= kErrIterCap;
        more = false;
    }
    if (more && global_ns() > ctl->t_deadline) {
        ctl->error |= kErrDeadline;
        more = false;
    }
    ctl->active = more ? 1u : 0u;
    if (p.use_cond) cudaGraphSetConditional(p.cond, more ? 1u : 0u);
    if (p.small_edges > 0) {
        ctl->small_run = ctl->in_edges <= (uint64_t)p.small_edges ? ctl->small_run + 1u : 0u;
        if (p.use_cond_small) cudaGraphSetConditional(p.cond_small, (more && ctl->small_run >= kSmallAfter) ? 1u : 0u);
    }
}

// Finalise a plain (non-HP) step: the output list becomes the input list.
// node_list: the output is a node / granule list needing a scan sentinel.
__device__ __forceinline__ void finish_plain_step(const StepParams &p, Ctl *ctl, bool node_list, int64_t cap) {
    __threadfence();
    const unsigned long long pk = ld_volatile(&ctl->out_pack);
    int64_t cnt = (int64_t)(pk >> 32);
    const int64_t edges = (int64_t)(pk & 0xFFFFFFFFull);
    if (cnt > cap) { ctl->error |= kErrCapacity; cnt = cap; }
    const int64_t step_edges = node_list ? (int64_t)ctl->in_edges : (int64_t)ctl->in_cnt;
    trace_append(ctl, kModeRelax, ctl->in_cnt, step_edges);
    ctl->relaxed += (unsigned long long)step_edges;
    const uint32_t out = ctl->par ^ 1u;
    if (node_list) p.lists[out].scan[cnt] = (int32_t)edges;
    ctl->par = out;
    ctl->in_cnt = (uint32_t)cnt;
    ctl->in_edges = (uint64_t)edges;
    ctl->out_pack = 0ull;
    ctl->level += 1;
    ctl->step += 1;
    ctl->blocks_done = 0;
    set_loop(p, ctl, cnt > 0);
    __threadfence();
}

// Tile size of an iteration over E list edges on `grid` CTAs: the smallest
// multiple of kTileGrain (at most max_tile) that still gives every CTA about
// two tiles, so small lists spread over the grid and large ones keep long
// tiles.
__device__ __forceinline__ int64_t iteration_tile(int64_t E, int64_t grid, int64_t max_tile) {
    const int64_t qmax = max_tile / kTileGrain > 0 ? max_tile / kTileGrain : 1;
    int64_t q = (E + kTileGrain * 2 * grid - 1) / (kTileGrain * 2 * grid);
    q = q < 1 ? 1 : (q > qmax ? qmax : q);
    return q * kTileGrain;
}

// Largest k in [lo, hi) with scan[k] <= e (read-only list, L1-cached).
__device__ __forceinline__ int64_t list_search(const int32_t *__restrict__ scan, int64_t lo, int64_t hi, int64_t e) {
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(scan + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace lbk
