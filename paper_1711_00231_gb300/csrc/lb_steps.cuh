// Step kernels: one launch = one worklist iteration (or one HP sub-step).
//
// Every kernel runs on a fixed, persistent-style grid (a multiple of the SM
// count) and reads the sizes of its input list from the device control
// block, so the same launch can be captured once into a CUDA graph and
// replayed by a conditional WHILE node until the worklist is empty.
#pragma once

#include <type_traits>

#include "lb_device.cuh"

// CTAs per SM the WD relax is compiled for (40 registers at 6, 48 at 5,
// 64 at 4), BFS and SSSP.  Measured on R-MAT scale 24 with the windowed
// walk and 3 edges per lane per round: BFS 2.08 / 2.19 / 2.48 ms at 6 / 5 /
// 4 CTAs, SSSP 9.37 / 9.39 / 10.6 ms; with deferred claims BFS 1.80 / 1.86
// ms at 6 / 5 CTAs and SSSP 7.70 / 7.52 ms.  SSSP now takes 4 edges per lane
// at 4 CTAs (6.70 -> 6.58 ms against 3 edges at 5 CTAs).
#ifndef LB_WD_MIN_BLOCKS
#define LB_WD_MIN_BLOCKS 6
#endif
#ifndef LB_WD_MIN_BLOCKS_SSSP
#define LB_WD_MIN_BLOCKS_SSSP 4
#endif
// Column and weight streams loaded evict-first (ld.global.cs) so the
// randomly read distance, queued and visited lines keep their place in L2
// (bit mask: 1 = SSSP, 2 = BFS).  Measured on R-MAT scale 24: SSSP 3.7%
// faster, BFS unchanged.
#ifndef LB_WD_STREAM
#define LB_WD_STREAM 3
#endif
template <bool SSSP, class T>
__device__ __forceinline__ T ld_edge(const T *p) {
    constexpr bool kStream = (LB_WD_STREAM & (SSSP ? 1 : 2)) != 0;
    return kStream ? __ldcs(p) : __ldg(p);
}

// 16-byte column / weight loads (bit mask: 1 = SSSP, 2 = BFS): with 4 edges
// per lane per group, a group that lies inside one adjacency list is read
// as one 16-byte load per lane and array (lane l takes the group's edges
// 4l .. 4l + 3).  A group starting off a 16-byte boundary is loaded from
// the boundary below with its first 1-3 edges masked, after which the rest
// of the list is aligned.  Used only when the arrays start on 16-byte
// boundaries (a custom allocator may return other addresses).
#ifndef LB_WD_VEC
#define LB_WD_VEC 0
#endif
template <bool SSSP, int R>
__host__ __device__ constexpr bool wd_vec() {
    return R == 4 && (LB_WD_VEC & (SSSP ? 1 : 2)) != 0;
}
template <bool SSSP, class T>
__device__ __forceinline__ uint4 ld_edge4(const T *p) {
    constexpr bool kStream = (LB_WD_STREAM & (SSSP ? 1 : 2)) != 0;
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    return kStream ? __ldcs(q) : __ldg(q);
}
__device__ __forceinline__ uint32_t u4_get(const uint4 &x, int r) {
    return r == 0 ? x.x : r == 1 ? x.y : r == 2 ? x.z : x.w;
}

// Push-buffer entries per warp of the WD step kernel (BFS, SSSP).  The
// shared-memory footprint decides the L1 carve-out left for the randomly
// read visited bitmap and distances.
#ifndef LB_KWB_WD_BFS
#define LB_KWB_WD_BFS 96
#endif
#ifndef LB_KWB_WD_SSSP
#define LB_KWB_WD_SSSP 128
#endif
// Deferred claims in the WD step kernel: the relax only buffers the
// candidates that pass the plain check, and the flush makes their atomics
// for a whole buffer at once (BFS: the visited-bit claim, FlushOut::defer
// == 2; SSSP: the atomicMin and the queued-bit claim, defer == 3).  The
// atomics then leave each relax group's chain of dependent accesses.
// Measured on R-MAT scale 24, 8 sources: BFS 1.93 -> 1.80 ms, SSSP 8.47
// -> 7.69 ms per query.
#ifndef LB_BFS_DEFER_CLAIM
#define LB_BFS_DEFER_CLAIM 1
#endif
#ifndef LB_SSSP_DEFER_CLAIM
#define LB_SSSP_DEFER_CLAIM 1
#endif

// Runs through long adjacency lists: after the first group of a run, the
// following groups of the same entry skip the window and bounds work, and
// (SSSP) a run of a stale entry is skipped whole (bit mask: 1 = SSSP, 2 =
// BFS).  Measured on R-MAT scale 24 with the bitmap at one address: SSSP
// 6.64 -> 6.16 ms per query, BFS 1% to 3% slower (not used).
#ifndef LB_WD_RUN_LOOP
#define LB_WD_RUN_LOOP 1
#endif
template <bool SSSP>
__host__ __device__ constexpr bool wd_run_loop() {
    return (LB_WD_RUN_LOOP & (SSSP ? 1 : 2)) != 0;
}
// SSSP: the walk skips the loads of entries whose vertex was queued again
// in this iteration (they relax nothing: the next iteration expands them).
// Measured on R-MAT scale 24: SSSP 7.38 -> 6.64 ms per query.
#ifndef LB_SSSP_SKIP_STALE
#define LB_SSSP_SKIP_STALE 1
#endif

// A warp's slice that starts on a tile-start grain takes its first list
// entry from the recorded tile starts instead of a warp-wide search (SSSP,
// and BFS in the persistent kernels).  Measured: R-MAT scale 24 SSSP 1.2%
// faster, 4096^2 grid BFS 2.6% and SSSP 4.4% faster; the single-level BFS
// step keeps the search (2% slower with the lookup: more spills).
#ifndef LB_WD_GRAIN_START
#define LB_WD_GRAIN_START 1
#endif
template <bool SSSP, bool COH>
__host__ __device__ constexpr bool wd_grain_start() {
    return LB_WD_GRAIN_START && (SSSP || COH);
}
// Deferred claims in the persistent small-list kernel (as in the WD step;
// bit mask: 1 = SSSP, 2 = BFS).  Measured on the 4096^2 grid: BFS equal,
// SSSP 2% slower with them (408 -> 416 ms), so BFS only.
#ifndef LB_SMALL_DEFER_CLAIM
#define LB_SMALL_DEFER_CLAIM 2
#endif

// The final flush of a WD iteration (and of a serving RELAX tile) as one
// list reservation per CTA (wflush_block) instead of one per warp.
#ifndef LB_BLOCK_FLUSH
#define LB_BLOCK_FLUSH 1
#endif

namespace lbk {

// ---------------------------------------------------------------------------
// Thread per worklist entry: BS (entries are whole nodes) and NS (entries
// are granules of at most MDT edges).  The edge loop is warp-uniform so the
// warp can push between edges; lanes whose entry is exhausted idle, which is
// exactly the load imbalance the node-based baseline exhibits (Sec. II-A).
// ---------------------------------------------------------------------------
template <bool SSSP, int OUTK>
__global__ void __launch_bounds__(kBlock) k_step_entry(StepParams p) {
    __shared__ WarpBuf s_wb[kWarps];
    __shared__ WarpScratch s_ws[kWarps];
    Ctl *ctl = p.ctl;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    uint32_t *status = ctl->status;
    const NodeList in = p.lists[par];
    FlushOut o;
    o.list = p.lists[par ^ 1u];
    o.elist = nullptr;
    o.pack = &ctl->out_pack;
    o.cap = p.list_cap;
    o.tile_cap = p.tile_cap;
    o.tile = (int32_t)kTileGrain;
    o.mdt = p.mdt;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    WarpBuf &wb = s_wb[warp];
    WarpScratch &ws = s_ws[warp];
    uint32_t cnt = 0;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t base = (int64_t)blockIdx.x * kBlock + warp * 32; base < in_cnt; base += stride) {
        const int64_t i = base + lane;
        int64_t cur = 0, end = 0;
        uint32_t du = 0;
        if (i < in_cnt) {
            cur = __ldg(in.beg + i);
            end = cur + (__ldg(in.scan + i + 1) - __ldg(in.scan + i));
            if (cur < 0 || end > p.g.m || cur > end) {
                atomicOr(&ctl->error, kErrBounds);
                cur = end = 0;
            } else if (SSSP) {
                du = sssp_source_dist(status, qcur, __ldg(in.v + i));
            }
        }
        while (__any_sync(kFull, cur < end)) {
            bool want = false;
            int32_t v = 0;
            int64_t vb = 0;
            uint32_t vd = 0;
            if (cur < end) {
                v = __ldg(p.g.col + cur);
                const bool hit = SSSP ? sssp_relax(status, qcur, v, du, __ldg(p.g.w + cur), ctl)
                                      : bfs_claim(p.bitmap, status, v, level + 1);
                if (hit) {
                    vb = __ldg(p.g.off + v);
                    vd = (uint32_t)(__ldg(p.g.off + v + 1) - vb);
                    want = vd > 0;
                }
                ++cur;
            }
            wpush(wb, cnt, want, v, vb, vd);
            if (cnt > kWB - 32) wflush<OUTK, false>(wb, ws, cnt, o);
        }
    }
    wflush<OUTK, false>(wb, ws, cnt, o);
    if (block_is_last(ctl) && threadIdx.x == 0) finish_plain_step(p, ctl, true, p.list_cap);
}

// ---------------------------------------------------------------------------
// Node splitting with physical child nodes (Sec. III-B and its listings): a
// node of out-degree d > MDT has ceil(d/MDT) - 1 children with ids n..n+S-1,
// each owning the next run of MDT of its edges; children have no in-edges.
// The parent's distance is reflected onto its children: whoever lowers a
// split node's distance also lowers its children's (the extra child-update
// atomics the paper lists as NS's cost), and an updated node is queued
// together with its children.  Thread per worklist entry, as in the
// node-based kernel.
// ---------------------------------------------------------------------------
template <bool SSSP>
__global__ void __launch_bounds__(kBlock) k_step_phys(StepParams p) {
    __shared__ WarpBuf s_wb[kWarps];
    __shared__ WarpScratch s_ws[kWarps];
    Ctl *ctl = p.ctl;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    uint32_t *status = ctl->status;
    const int64_t n = p.g.n;
    const NodeList in = p.lists[par];
    FlushOut o;
    o.list = p.lists[par ^ 1u];
    o.elist = nullptr;
    o.pack = &ctl->out_pack;
    o.cap = p.list_cap;
    o.tile_cap = p.tile_cap;
    o.tile = (int32_t)kTileGrain;
    o.mdt = p.mdt;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    o.child_first = p.child_first;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    WarpBuf &wb = s_wb[warp];
    WarpScratch &ws = s_ws[warp];
    uint32_t cnt = 0;
    const int64_t mdt = p.mdt;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t base = (int64_t)blockIdx.x * kBlock + warp * 32; base < in_cnt; base += stride) {
        const int64_t i = base + lane;
        int64_t cur = 0, end = 0;
        uint32_t du = 0;
        if (i < in_cnt) {
            cur = __ldg(in.beg + i);
            end = cur + (__ldg(in.scan + i + 1) - __ldg(in.scan + i));
            const int32_t x = __ldg(in.v + i);
            if (cur < 0 || end > p.g.m || cur > end || x < 0 || (int64_t)x >= n + p.n_children) {
                atomicOr(&ctl->error, kErrBounds);
                cur = end = 0;
            } else if (SSSP) {
                if ((int64_t)x < n) {
                    du = sssp_source_dist(status, qcur, x);
                } else {
                    const int32_t parent = __ldg(p.parent_of + (x - n));
                    du = is_queued<false>(qcur, parent) ? kInf : p.child_dist[x - n];
                }
            }
        }
        while (__any_sync(kFull, cur < end)) {
            bool want = false;
            int32_t v = 0;
            int64_t vb = 0;
            uint32_t vd = 0;
            if (cur < end) {
                v = __ldg(p.g.col + cur);
                if (SSSP) {
                    const uint64_t a64 = (uint64_t)du + (uint64_t)__ldg(p.g.w + cur);
                    const uint32_t alt = du == kInf ? kInf : (a64 >= kSat ? kSat : (uint32_t)a64);
                    if (alt < status[v]) {
                        const uint32_t old = atomicMin(&status[v], alt);
                        if (alt < old) {
                            if (alt == kSat) atomicOr(&ctl->error, kErrSaturated);
                            vb = __ldg(p.g.off + v);
                            vd = (uint32_t)(__ldg(p.g.off + v + 1) - vb);
                            const int32_t cf = __ldg(p.child_first + v);
                            if (cf >= 0) {
                                const int64_t nk = ((int64_t)vd + mdt - 1) / mdt - 1;
                                for (int64_t c = 0; c < nk; ++c) atomicMin(&p.child_dist[cf - n + c], alt);
                            }
                            want = vd > 0 && !is_queued<false>(qcur, v) &&
                                   !(atomicOr(&qcur[(uint32_t)v >> 5], 1u << ((uint32_t)v & 31u)) &
                                     (1u << ((uint32_t)v & 31u)));
                        }
                    }
                } else if (bfs_claim(p.bitmap, status, v, level + 1)) {
                    vb = __ldg(p.g.off + v);
                    vd = (uint32_t)(__ldg(p.g.off + v + 1) - vb);
                    const int32_t cf = __ldg(p.child_first + v);
                    if (cf >= 0) {
                        const int64_t nk = ((int64_t)vd + mdt - 1) / mdt - 1;
                        for (int64_t c = 0; c < nk; ++c) p.child_dist[cf - n + c] = level + 1;
                    }
                    want = vd > 0;
                }
                ++cur;
            }
            wpush(wb, cnt, want, v, vb, vd);
            if (cnt > kWB - 32) wflush<kOutPhys, false>(wb, ws, cnt, o);
        }
    }
    wflush<kOutPhys, false>(wb, ws, cnt, o);
    if (block_is_last(ctl) && threadIdx.x == 0) finish_plain_step(p, ctl, true, p.list_cap);
}

// ---------------------------------------------------------------------------
// Workload decomposition (Sec. III-A) over CTA tiles.  The input list's
// edges (in list order) are cut into tiles of T edges; the push that built
// the list recorded the entry holding every kTileGrain-th list edge, so tile
// t starts in entry tstart[t * T / kTileGrain] (the paper's NodeOffset /
// EdgeOffset, found without a scan or an offset kernel).  Each warp takes a
// contiguous slice of T / 8 edges and walks it, so consecutive lanes read
// consecutive edges of a node (coalesced).  One warp-wide 32-way search per
// warp and tile finds the entry of the slice's first edge; after that the
// warp keeps the current entry in registers and a look-ahead window of the
// next 32 entries' prefix and first edge (one per lane, reloaded only when
// the walk advances).  Where the current entry reaches past the next 32
// edges the warp runs through it with plain strided loads; elsewhere a
// boundary step takes 32 edges: an entry starting inside the 32-edge window
// sets one bit of a mask (entries have at least one edge, so at most 32
// start in 32 positions); a lane's entry is the current one plus the number
// of starts at or before its position, and its prefix / first edge come
// from the loading lane by shuffle.  That replaces a per-edge search by a
// few warp-wide operations per 32 edges.
template <bool COH, class T>
__device__ __forceinline__ T ld_list(const T *p) {
    return COH ? __ldcg(p) : __ldg(p);
}

// The list entry holding list edge w0 within [lo, hi) (scan[lo] <= w0 <
// scan[hi], hi may be the end): a warp-wide 32-way search, 31 probes per
// round and a ballot, so a range of up to 32^k entries takes k rounds of
// one load latency each instead of k * 5 dependent loads.
template <bool COH, class IT, class KT>
__device__ __forceinline__ KT warp_search(const int32_t *scan, KT lo, KT hi, IT w0, uint32_t lane) {
    while (hi - lo > 1) {  // warp-uniform
        const KT step = (hi - lo + 31) / 32;
        const KT p = lo + step * (KT)(lane + 1);
        const bool le = p < hi && (IT)ld_list<COH>(scan + p) <= w0;
        const KT n = (KT)__popc(__ballot_sync(kFull, le));  // probes are increasing: a prefix of lanes
        lo += step * n;
        if (lo + step < hi) hi = lo + step;
    }
    return lo;
}

// The walk of one tile with a 64-entry window of the list in registers.
// Lane l holds entries kb + l and kb + 32 + l: the entry's first list edge
// s, the delta d = first CSR edge - s (an edge's CSR index is d + list
// edge) and, for SSSP, the distance du its edges relax with (kInf when the
// entry's node has been queued again in this iteration: the next one
// expands it with the newer value).  The current entry kcur stays within
// the window's first half, and the window slides by 32 entries when kcur
// leaves it: one reload per 32 entries, not per step.  A group of R x 32
// edges that lies inside entry kcur is loaded directly; otherwise each
// 32-edge step finds every lane's entry from the bit mask of entry starts
// inside the step (an entry has at least one edge, so at most 32 start in
// 32 positions) and takes its fields from the window by shuffle.  32-bit
// list edges and edge ids (< 2^31, checked when the graph is created).
template <bool SSSP, int R, bool COH, class WB, class WS>
__device__ __forceinline__ void wd_walk_win(const GraphDev &g, const NodeList &in, int64_t in_cnt, int64_t E,
                                            int64_t T, int64_t t, uint32_t *bitmap, uint32_t *qcur,
                                            uint32_t *status, uint32_t level, uint32_t *err, WB &wb,
                                            WS &ws, uint32_t &cnt, const FlushOut &o) {
    const int64_t q = T / kTileGrain;
    const int64_t W = T / kWarps;  // edges per warp and tile (a multiple of 32)
    const int64_t ntiles = (E + T - 1) / T;
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    const int64_t e0 = t * T;
    const int64_t e1 = min(e0 + T, E);
    const int64_t w064 = e0 + (int64_t)warp * W;
    if (w064 >= e1) return;  // warp-uniform
    const int32_t w0 = (int32_t)w064;
    // A slice that starts on a tile-start grain (every slice of a tile of
    // a multiple of 8 x 256 edges) takes its first entry from the tile
    // starts the push recorded; the load is issued with the tile's bounds.
    const bool on_grain = wd_grain_start<SSSP, COH>() && (w0 & (int32_t)(kTileGrain - 1)) == 0;
    const int32_t kg = on_grain ? ld_list<COH>(in.tstart + (w0 >> 8)) : 0;
    const int64_t i0 = ld_list<COH>(in.tstart + t * q);
    const int64_t ihi =
        (t + 1 < ntiles) ? min((int64_t)ld_list<COH>(in.tstart + (t + 1) * q) + 1, in_cnt) : in_cnt;
    if (i0 < 0 || i0 >= ihi) {
        if (lane == 0) atomicOr(err, kErrBounds);
        return;
    }
    const int32_t w1 = (int32_t)min(w064 + W, e1);
    const int32_t ihiK = (int32_t)ihi;
    const int32_t m = (int32_t)g.m;
    const bool vec_ok = wd_vec<SSSP, R>() &&
                        ((reinterpret_cast<uintptr_t>(g.col) | (SSSP ? reinterpret_cast<uintptr_t>(g.w) : 0u)) &
                         15u) == 0;
    int32_t kcur;
    if (on_grain) {
        if (kg < (int32_t)i0 || kg >= ihiK) {
            if (lane == 0) atomicOr(err, kErrBounds);
            return;
        }
        kcur = kg;
    } else {
        kcur = warp_search<COH, uint32_t, int32_t>(in.scan, (int32_t)i0, ihiK, (uint32_t)w0, lane);
    }
    int32_t kb = kcur;
    int32_t s0 = INT32_MAX, d0 = 0, s1 = INT32_MAX, d1 = 0;
    uint32_t u0 = kInf, u1 = kInf;  // SSSP: distance the entry relaxes with
    auto load = [&](int32_t j, int32_t &sj, int32_t &dj, uint32_t &uj) {
        sj = INT32_MAX;
        dj = 0;
        uj = kInf;
        if (j < ihiK) {
            sj = ld_list<COH>(in.scan + j);
            dj = ld_list<COH>(in.beg + j) - sj;
            if (SSSP) {
                const int32_t u = ld_list<COH>(in.v + j);
                if (u >= 0 && (int64_t)u < g.n) uj = is_queued<COH>(qcur, u) ? kInf : ld_mut<COH>(status + u);
            }
        }
    };
    load(kb + (int32_t)lane, s0, d0, u0);
    load(kb + 32 + (int32_t)lane, s1, d1, u1);
    int32_t ew = w0;
    // the run in progress (wd_run_loop): its CSR delta, the list edge where
    // its entry ends and where the warp's slice or the entry ends (0:
    // none), and (SSSP) the distance it relaxes with
    int32_t run_d = 0, run_next = 0, run_end = 0;
    uint32_t run_du = 0u;
    while (ew < w1) {  // warp-uniform
        bool ok[R];
        int32_t vv[R];
        uint32_t ww[R], dd[R];
        if (wd_run_loop<SSSP>() && ew + 32 * R <= run_end) {
            // a further group of the run: no window or bounds work
            if (wd_vec<SSSP, R>() && vec_ok && ((run_d + ew) & 3) == 0) {
                const int32_t a = run_d + ew + 4 * (int32_t)lane;
                const uint4 c4 = ld_edge4<SSSP>(g.col + a);
                const uint4 w4 = SSSP ? ld_edge4<SSSP>(g.w + a) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    ok[r] = true;
                    vv[r] = (int32_t)u4_get(c4, r);
                    ww[r] = u4_get(w4, r);
                    dd[r] = SSSP ? run_du : 0u;
                }
                ew += 32 * R;
                if (run_next == ew) kcur += 1;
                goto relax_group;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int32_t e = ew + 32 * r + (int32_t)lane;
                ok[r] = true;
                vv[r] = ld_edge<SSSP>(g.col + (run_d + e));
                ww[r] = SSSP ? ld_edge<SSSP>(g.w + (run_d + e)) : 0u;
                dd[r] = SSSP ? run_du : 0u;
            }
            ew += 32 * R;
            if (run_next == ew) kcur += 1;
            goto relax_group;
        }
        if (kcur >= kb + 32) {  // slide: the second half becomes the first
            kb += 32;
            s0 = s1;
            d0 = d1;
            u0 = u1;
            load(kb + 32 + (int32_t)lane, s1, d1, u1);
        }
        {
        // start of entry kcur + 1 (window position 1..32)
        const int32_t pn = kcur + 1 - kb;
        const int32_t s_next = __shfl_sync(kFull, pn < 32 ? s0 : s1, pn & 31);
        if (s_next >= ew + 32 * R) {
            // the whole group lies inside entry kcur
            const int32_t pc = kcur - kb;
            const int32_t dcur = __shfl_sync(kFull, d0, pc);
            const uint32_t ducur = SSSP ? __shfl_sync(kFull, u0, pc) : 0u;
            if (wd_run_loop<SSSP>()) {
                // the whole run is checked once
                if (dcur + ew < 0 || dcur + min(s_next, w1) > m) {
                    if (lane == 0) atomicOr(err, kErrBounds);
                    return;
                }
                if (SSSP && LB_SSSP_SKIP_STALE && ducur == kInf) {
                    // queued again in this iteration: the entry relaxes nothing
                    ew = min(s_next, w1);
                    if (s_next == ew) kcur += 1;
                    continue;
                }
                run_d = dcur;
                run_next = s_next;
                run_end = min(s_next, w1);
                if (SSSP) run_du = ducur;
            } else if (dcur + ew < 0 || dcur + min(ew + 32 * R, w1) > m) {
                if (lane == 0) atomicOr(err, kErrBounds);
                return;
            }
            if (wd_vec<SSSP, R>() && vec_ok && ew + 32 * R <= w1) {
                // 16-byte loads from the boundary at or below the group's
                // first edge; the h edges before it are masked and the
                // group takes 32 R - h edges (so later groups are aligned).
                // [dcur + ew - h, dcur + ew + 32 R - h) lies inside the
                // checked range [dcur + ew, dcur + w1) widened by h < 4
                // edges of this list's predecessors, all below m.
                const int32_t h = (dcur + ew) & 3;
                const int32_t a = dcur + ew - h + 4 * (int32_t)lane;
                const bool live = !SSSP || !LB_SSSP_SKIP_STALE || ducur != kInf;
                uint4 c4 = make_uint4(0u, 0u, 0u, 0u), w4 = make_uint4(0u, 0u, 0u, 0u);
                if (live) {
                    c4 = ld_edge4<SSSP>(g.col + a);
                    if (SSSP) w4 = ld_edge4<SSSP>(g.w + a);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    ok[r] = live && 4 * (int32_t)lane + r >= h;
                    vv[r] = (int32_t)u4_get(c4, r);
                    ww[r] = u4_get(w4, r);
                    dd[r] = ducur;
                }
                ew += 32 * R - h;
                if (s_next == ew) kcur += 1;
                goto relax_group;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int32_t e = ew + 32 * r + (int32_t)lane;
                // SSSP: an entry queued again in this iteration (ducur =
                // kInf) relaxes nothing; its edges are not loaded
                ok[r] = e < w1 && (!SSSP || !LB_SSSP_SKIP_STALE || ducur != kInf);
                vv[r] = ok[r] ? ld_edge<SSSP>(g.col + (dcur + e)) : 0;
                ww[r] = (SSSP && ok[r]) ? ld_edge<SSSP>(g.w + (dcur + e)) : 0u;
                dd[r] = ducur;
            }
            ew += 32 * R;
            if (s_next == ew) kcur += 1;
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ok[r] = false;
                vv[r] = 0;
                ww[r] = 0u;
                dd[r] = 0u;
                if (ew >= w1) continue;  // warp-uniform
                if (kcur >= kb + 32) {
                    kb += 32;
                    s0 = s1;
                    d0 = d1;
                    u0 = u1;
                    load(kb + 32 + (int32_t)lane, s1, d1, u1);
                }
                // bit p - 1 of `starts`: an entry starts at ew + p, for p = 1..32
                // (entries have at least one edge, so at most 32 start there)
                const int32_t p0 = s0 - ew - 1, p1 = s1 - ew - 1;
                const uint32_t bits = ((uint32_t)p0 < 32u ? (1u << p0) : 0u) | ((uint32_t)p1 < 32u ? (1u << p1) : 0u);
                const uint32_t starts = __reduce_or_sync(kFull, bits);
                const int32_t pe = kcur - kb + __popc(starts & lanemask_lt());  // window position of my entry
                const int32_t x0 = __shfl_sync(kFull, d0, pe & 31);
                const int32_t x1 = __shfl_sync(kFull, d1, pe & 31);
                uint32_t du = 0u;
                if (SSSP) {
                    const uint32_t y0 = __shfl_sync(kFull, u0, pe & 31);
                    const uint32_t y1 = __shfl_sync(kFull, u1, pe & 31);
                    du = pe < 32 ? y0 : y1;
                }
                const int32_t e = ew + (int32_t)lane;
                const int32_t eidx = (pe < 32 ? x0 : x1) + e;
                if (e < w1 && (!SSSP || !LB_SSSP_SKIP_STALE || du != kInf)) {
                    if ((uint32_t)eidx >= (uint32_t)m) {
                        atomicOr(err, kErrBounds);
                    } else {
                        ok[r] = true;
                        vv[r] = ld_edge<SSSP>(g.col + eidx);
                        if (SSSP) {
                            ww[r] = ld_edge<SSSP>(g.w + eidx);
                            dd[r] = du;
                        }
                    }
                }
                // the entry holding the next step's first edge
                kcur += __popc(starts);
                ew += 32;
            }
        }
        }
    relax_group:
        if constexpr (SSSP) {
            if (o.defer == 3) {
                relax_sssp_defer<R, COH>(ok, vv, ww, dd, status, wb, ws, cnt, o);
                continue;
            }
            if (cnt > WB::kCap - 32 * R) wflush<kOutNode, true>(wb, ws, cnt, o);
            relax_items<true, R, kOutNode, true, COH, false>(ok, vv, ww, dd, g.off, bitmap, qcur, status, level, err,
                                                             wb, ws, cnt, o);
        } else {
            relax_bfs_lean<R, COH>(ok, vv, g.off, bitmap, status, level, wb, ws, cnt, o);
        }
    }
}

// One tile of the walk.  COH selects L2-coherent loads for everything other
// CTAs write (the persistent serving and small-list kernels); the
// single-level launches use the read-only / L1 paths.
template <bool SSSP, int STEPS, bool COH, class WB, class WS>
__device__ __forceinline__ void wd_walk_tile(const GraphDev &g, const NodeList &in, int64_t in_cnt, int64_t E,
                                             int64_t T, int64_t t, uint32_t *bitmap, uint32_t *qcur,
                                             uint32_t *status, uint32_t level, uint32_t *err, WB &wb,
                                             WS &ws, uint32_t &cnt, const FlushOut &o) {
    wd_walk_win<SSSP, STEPS, COH>(g, in, in_cnt, E, T, t, bitmap, qcur, status, level, err, wb, ws, cnt, o);
}

template <bool SSSP, int STEPS, class WB, class WS>
__device__ __forceinline__ void wd_walk(const StepParams &p, Ctl *ctl, const NodeList &in, int64_t in_cnt, int64_t E,
                                        WB &wb, WS &ws, uint32_t &cnt, const FlushOut &o,
                                        uint32_t *status, uint32_t level, uint32_t *qcur) {
    const int64_t T = iteration_tile(E, gridDim.x, p.tile);
    const int64_t ntiles = (E + T - 1) / T;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
        wd_walk_tile<SSSP, STEPS, false>(p.g, in, in_cnt, E, T, t, p.bitmap, qcur, status, level,
                                         &ctl->error, wb, ws, cnt, o);
}

template <bool SSSP, int ITEMS>
__global__ void __launch_bounds__(kBlock, SSSP ? LB_WD_MIN_BLOCKS_SSSP : LB_WD_MIN_BLOCKS) k_step_wd(StepParams p) {
    // node pushes only: no flush scratch
    __shared__ WarpBufT<SSSP ? LB_KWB_WD_SSSP : LB_KWB_WD_BFS> s_wb[kWarps];
    NoScratch ns;
    Ctl *ctl = p.ctl;
    // the small-list kernel that runs before this step in the device loop
    // may have finished the query (uniform: every CTA reads the same flag)
    if (p.small_edges > 0 && ctl->active == 0u) return;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const int64_t E = (int64_t)ctl->in_edges;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    uint32_t *status = ctl->status;
    const NodeList in = p.lists[par];
    FlushOut o;
    o.list = p.lists[par ^ 1u];
    o.elist = nullptr;
    o.pack = &ctl->out_pack;
    o.cap = p.list_cap;
    o.tile_cap = p.tile_cap;
    o.tile = (int32_t)kTileGrain;
    o.mdt = p.mdt;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    o.off = p.g.off;
    o.defer = SSSP ? (LB_SSSP_DEFER_CLAIM ? 3 : LB_DEFER_OFFSETS) : (LB_BFS_DEFER_CLAIM ? 2 : LB_DEFER_OFFSETS);
    o.claim_bitmap = SSSP ? qcur : p.bitmap;
    o.claim_status = status;
    o.claim_level = level;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t cnt = 0;
    wd_walk<SSSP, ITEMS>(p, ctl, in, in_cnt, E, s_wb[warp], ns, cnt, o, status, level, qcur);
#if LB_BLOCK_FLUSH
    wflush_block<kOutNode, true>(s_wb[warp], ns, cnt, o);
#else
    wflush<kOutNode, true>(s_wb[warp], ns, cnt, o);
#endif
    if (block_is_last(ctl) && threadIdx.x == 0) finish_plain_step(p, ctl, true, p.list_cap);
}

// ---------------------------------------------------------------------------
// Small-list levels in one persistent launch (WD).  A high-diameter graph
// (a grid: thousands of levels of a few thousand edges) spends most of a
// level on the launch and the end-of-step protocol, not on edges.  While
// the input list has at most p.small_edges edges, this kernel (one CTA per
// SM, launched cooperatively so that every CTA is resident) runs level
// after level: the workload-decomposition walk over the list, a block-wide
// flush into the output list, then a grid barrier, after which every CTA
// reads the output list's size and continues with it.  It leaves the loop
// state in the control block when the list empties, grows past the limit,
// or a cap is reached; the regular WD step runs the large levels.  Level L
// counts its pushes in small_pack[L % 3]; CTA 0 zeroes the counter of level
// L + 1 during level L (its last reads were right after the barrier ending
// level L - 2, and every CTA has passed the barrier ending level L - 1
// since), and all three after a last barrier before the launch returns, so
// they start at zero in every launch.  Data other CTAs write during the
// launch is read through L2.
// The barrier's wait is bounded: after kBarrierLimitNs a CTA records
// kErrDeadline, ends the device loop and returns, so a barrier that cannot
// complete ends the query with LB_ERR_TIMEOUT instead of a hang.
constexpr uint64_t kBarrierLimitNs = 2000000000ull;

// Grid barrier among the launch's CTAs (every thread calls it).  Returns
// false when the wait ran past kBarrierLimitNs; *stop receives the
// releasing CTA's verdict on the query's time limit.
__device__ __forceinline__ bool grid_barrier(Ctl *ctl, bool *stop) {
    __shared__ uint32_t s_ok, s_stop;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gen = *(volatile uint32_t *)&ctl->bar_gen;
        __threadfence();
        const uint32_t arrived = atomicAdd(&ctl->bar_count, 1u);
        uint32_t ok = 1u;
        if (arrived == gridDim.x - 1) {
            ctl->bar_count = 0u;
            ctl->bar_stop = global_ns() > ctl->t_deadline ? 1u : 0u;
            __threadfence();
            atomicExch(&ctl->bar_gen, gen + 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*(volatile uint32_t *)&ctl->bar_gen == gen) {
                if (global_ns() - t0 > kBarrierLimitNs) {
                    ok = 0u;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
        s_stop = *(volatile uint32_t *)&ctl->bar_stop;
    }
    __syncthreads();
    *stop = s_stop != 0u;
    return s_ok != 0u;
}

#ifndef LB_SMALL_CTAS
#define LB_SMALL_CTAS 1
#endif
template <bool SSSP, int ITEMS>
__global__ void __launch_bounds__(kBlock, LB_SMALL_CTAS) k_small_levels(StepParams p) {
    // node pushes only: no flush scratch
    __shared__ WarpBuf s_wb[kWarps];
    NoScratch ns;
    Ctl *ctl = p.ctl;
    const int64_t lim = p.small_edges;
    uint32_t level = *(volatile uint32_t *)&ctl->level;
    uint32_t par = *(volatile uint32_t *)&ctl->par;
    int64_t in_cnt = *(volatile uint32_t *)&ctl->in_cnt;
    int64_t E = (int64_t)*(volatile uint64_t *)&ctl->in_edges;
    // uniform: every CTA reads the same state left by the previous launch
    if (lim <= 0 || *(volatile uint32_t *)&ctl->active == 0u || in_cnt == 0 || E > lim ||
        *(volatile uint32_t *)&ctl->small_run < kSmallAfter)
        return;
    uint32_t *status = ctl->status;
    const uint32_t warp = threadIdx.x >> 5;
    const uint64_t step0 = ctl->step;
    const uint32_t max_levels = ctl->max_levels;
    uint64_t steps = 0;
    bool failed = false;
    for (;;) {
        uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
        const NodeList in = p.lists[par];
        if (SSSP) {
            // the other half holds the bits of the previous level, whose queued
            // vertices with out-edges are exactly this level's entries (bits of
            // vertices without out-edges are never read): clear those
            uint32_t *qn = queued_half(p.bitmap, p.bm_words, level + 1u);
            const int64_t stride = (int64_t)gridDim.x * blockDim.x;
            for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < in_cnt; k += stride) {
                const int32_t u = __ldcg(in.v + k);
                if (u >= 0 && (int64_t)u < p.g.n) atomicAnd(&qn[(uint32_t)u >> 5], ~(1u << ((uint32_t)u & 31u)));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->small_pack[(level + 1u) % 3u] = 0ull;
        FlushOut o;
        o.list = p.lists[par ^ 1u];
        o.elist = nullptr;
        o.pack = &ctl->small_pack[level % 3u];
        o.cap = p.list_cap;
        o.tile_cap = p.tile_cap;
        o.tile = (int32_t)kTileGrain;
        o.mdt = p.mdt;
        o.err = &ctl->error;
        o.pushes = &ctl->pushes;
        o.child_first = nullptr;
        o.off = p.g.off;
        o.defer = SSSP ? ((LB_SMALL_DEFER_CLAIM & 1) ? 3 : LB_DEFER_OFFSETS)
                       : ((LB_SMALL_DEFER_CLAIM & 2) ? 2 : LB_DEFER_OFFSETS);
        o.claim_bitmap = SSSP ? qcur : p.bitmap;
        o.claim_status = status;
        o.claim_level = level;
        uint32_t cnt = 0;
        const int64_t T = iteration_tile(E, gridDim.x, p.tile);
        const int64_t ntiles = (E + T - 1) / T;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
            wd_walk_tile<SSSP, ITEMS, true>(p.g, in, in_cnt, E, T, t, p.bitmap, qcur, status, level, &ctl->error,
                                            s_wb[warp], ns, cnt, o);
        wflush_block<kOutNode, true>(s_wb[warp], ns, cnt, o);
        // test hook: one CTA that never arrives makes the others' waits run out
        if (p.test_barrier_skip && blockIdx.x == 1) return;
        bool stop = false;
        if (!grid_barrier(ctl, &stop)) {
            failed = true;
            break;
        }
        const unsigned long long pk = __ldcg(&ctl->small_pack[level % 3u]);
        int64_t ncnt = (int64_t)(pk >> 32);
        const int64_t nedges = (int64_t)(pk & 0xFFFFFFFFull);
        if (ncnt > p.list_cap) {
            if (threadIdx.x == 0) atomicOr(&ctl->error, kErrCapacity);
            ncnt = p.list_cap;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const uint32_t tl = ctl->trace_len;
            if (tl < (uint32_t)kTraceMax) {
                ctl->trace[tl].level = (int32_t)level;
                ctl->trace[tl].mode = kModeSmall;
                ctl->trace[tl].list_size = in_cnt;
                ctl->trace[tl].edges = E;
                ctl->trace[tl].t_ns = (int64_t)(global_ns() - ctl->t_start);
                ctl->trace_len = tl + 1;
            }
            ctl->relaxed += (unsigned long long)E;
        }
        par ^= 1u;
        level += 1u;
        in_cnt = ncnt;
        E = nedges;
        ++steps;
        if (stop || in_cnt == 0 || E > lim || level >= max_levels) break;
    }
    // every CTA has read its last counter before CTA 0 zeroes them
    bool stop_unused = false;
    if (!failed && !grid_barrier(ctl, &stop_unused)) failed = true;
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(&ctl->error, kErrDeadline);
            ctl->active = 0u;
            if (p.use_cond) cudaGraphSetConditional(p.cond, 0u);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) ctl->small_pack[k] = 0ull;
        p.lists[par].scan[in_cnt] = (int32_t)E;  // sentinel (read by other strategies' kernels)
        ctl->par = par;
        ctl->level = level;
        ctl->in_cnt = (uint32_t)in_cnt;
        ctl->in_edges = (uint64_t)E;
        ctl->out_pack = 0ull;
        ctl->step = step0 + steps;
        set_loop(p, ctl, in_cnt > 0);
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// Edge-based distribution (Sec. II-B): one thread per worklist edge of the
// COO graph (source from coo_src, destination and weight from the CSR
// arrays, which double as the COO dst / wt arrays).  An updated node pushes
// all of its edge ids with one reservation (work chunking).
// ---------------------------------------------------------------------------
template <bool SSSP, int ITEMS, bool CHUNK>
__global__ void __launch_bounds__(kBlock) k_step_ep(StepParams p) {
    __shared__ WarpBuf s_wb[kWarps];
    __shared__ WarpScratch s_ws[kWarps];
    Ctl *ctl = p.ctl;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    uint32_t *status = ctl->status;
    const int32_t *in = p.elist[par];
    FlushOut o;
    o.list = p.lists[0];
    o.elist = p.elist[par ^ 1u];
    o.pack = &ctl->out_pack;
    o.cap = p.elist_cap;
    o.tile_cap = 0;
    o.tile = (int32_t)kTileGrain;
    o.mdt = p.mdt;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    const uint32_t warp = threadIdx.x >> 5;
    WarpBuf &wb = s_wb[warp];
    WarpScratch &ws = s_ws[warp];
    uint32_t cnt = 0;
    const int64_t chunk = (int64_t)kBlock * ITEMS;
    for (int64_t r0 = (int64_t)blockIdx.x * chunk; r0 < in_cnt; r0 += (int64_t)gridDim.x * chunk) {
        int32_t vv[ITEMS];
        uint32_t ww[ITEMS], dd[ITEMS];
        bool ok[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const int64_t i = r0 + (int64_t)it * kBlock + threadIdx.x;
            ok[it] = i < in_cnt;
            vv[it] = 0;
            ww[it] = 0;
            dd[it] = 0;
            if (ok[it]) {
                const int32_t e = __ldg(in + i);
                if (e < 0 || (int64_t)e >= p.g.m) {
                    atomicOr(&ctl->error, kErrBounds);
                    ok[it] = false;
                    continue;
                }
                vv[it] = __ldg(p.g.col + e);
                if (SSSP) {
                    ww[it] = __ldg(p.g.w + e);
                    dd[it] = sssp_source_dist(status, qcur, __ldg(p.coo_src + e));
                }
            }
        }
        relax_items<SSSP, ITEMS, CHUNK ? kOutEdges : kOutEdgesPerEdge, false>(
            ok, vv, ww, dd, p.g.off, p.bitmap, qcur, status, level, &ctl->error, wb, ws, cnt, o);
    }
    wflush<kOutEdges, false>(wb, ws, cnt, o);
    if (block_is_last(ctl) && threadIdx.x == 0) finish_plain_step(p, ctl, false, p.elist_cap);
}

// ---------------------------------------------------------------------------
// Hierarchical processing (Sec. III-C).  One launch is one step of the
// super-iteration: either a sub-iteration over the current list (each entry
// relaxes at most MDT edges; entries with edges left are pushed, with their
// remaining range, to the next sub-list) or, when the list is shorter than
// the threshold, one workload-decomposition step over everything left.
// Nodes updated in any step go to the next super worklist.
// ---------------------------------------------------------------------------
// Edges first + lane + k * stride (< last) of one node, relaxed ITEMS per
// lane at a time from source distance du (the warp and CTA bins of the
// degree-binned HP step).  first, last and stride are warp-uniform.
template <bool SSSP, int ITEMS, int OUTK = kOutNode, bool TILED = true>
__device__ __forceinline__ void serve_range(const StepParams &p, Ctl *ctl, int64_t first, int64_t last, int64_t stride,
                                            uint32_t du, uint32_t *status, uint32_t level, uint32_t *qcur,
                                            WarpBuf &wb, WarpScratch &ws, uint32_t &cnt, const FlushOut &o) {
    const uint32_t lane = lane_id();
    for (int64_t e0 = first; e0 < last; e0 += stride * ITEMS) {
        bool ok[ITEMS];
        int32_t vv[ITEMS];
        uint32_t ww[ITEMS], dd[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const int64_t e = e0 + (int64_t)it * stride + lane;
            ok[it] = e < last;
            vv[it] = ok[it] ? __ldg(p.g.col + e) : 0;
            ww[it] = (SSSP && ok[it]) ? __ldg(p.g.w + e) : 0u;
            dd[it] = du;
        }
        if (cnt > kWB - 32 * ITEMS) wflush<OUTK, TILED>(wb, ws, cnt, o);
        relax_items<SSSP, ITEMS, OUTK, TILED, false, false>(ok, vv, ww, dd, p.g.off, p.bitmap, qcur, status, level,
                                                           &ctl->error, wb, ws, cnt, o);
    }
}

// The degree-binned step (HP's hp_mode 1 and NS's ns_mode 1): every entry
// of the list is served in this one step at its own granularity -- an
// entry of at most tmax edges by its own thread, one of at most
// hp_warp_max edges by its warp (the warp takes its warp-class entries one
// after another), a larger one by the whole CTA after the block's batches
// (the CTA bin is a block-local list; when it is full the warp serves the
// entry instead).  OUTK / TILED: what the pushes write (nodes with tile
// starts for HP, granules for NS).  Every thread of the block calls it.
template <bool SSSP, int ITEMS, int OUTK, bool TILED>
__device__ __forceinline__ void binned_step(const StepParams &p, Ctl *ctl, const NodeList &in, int64_t in_cnt,
                                            int64_t tmax, uint32_t *status, uint32_t level, uint32_t *qcur,
                                            WarpBuf &wb, WarpScratch &ws, uint32_t &cnt, const FlushOut &o) {
    constexpr int kBigCap = 256;
    __shared__ int32_t s_big[kBigCap];
    __shared__ uint32_t s_nbig;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const int64_t wmax = p.hp_warp_max;
    const int64_t stride = (int64_t)gridDim.x * kBlock;
    for (int64_t base = (int64_t)blockIdx.x * kBlock + warp * 32; base < in_cnt; base += stride) {
        const int64_t i = base + lane;
        int64_t cur = 0, len = 0;
        uint32_t du = 0;
        int cls = -1;  // -1 nothing to do, 0 thread, 1 warp, 2 CTA
        if (i < in_cnt) {
            cur = __ldg(in.beg + i);
            len = __ldg(in.scan + i + 1) - __ldg(in.scan + i);
            if (cur < 0 || len < 0 || cur + len > p.g.m) {
                atomicOr(&ctl->error, kErrBounds);
            } else {
                if (SSSP) du = sssp_source_dist(status, qcur, __ldg(in.v + i));
                if (!SSSP || du != kInf) cls = len <= tmax ? 0 : (len <= wmax ? 1 : 2);
            }
        }
        if (cls == 2) {
            const uint32_t slot = atomicAdd(&s_nbig, 1u);
            if (slot < (uint32_t)kBigCap) s_big[slot] = (int32_t)i;
            else cls = 1;
        }
        unsigned wm = __ballot_sync(kFull, cls == 1);
        while (wm) {
            const int l = __ffs(wm) - 1;
            wm &= wm - 1;
            const int64_t c0 = __shfl_sync(kFull, cur, l);
            const int64_t n0 = __shfl_sync(kFull, len, l);
            const uint32_t d0 = __shfl_sync(kFull, du, l);
            serve_range<SSSP, ITEMS, OUTK, TILED>(p, ctl, c0, c0 + n0, 32, d0, status, level, qcur, wb, ws, cnt, o);
        }
        int64_t end = cls == 0 ? cur + len : cur;
        while (__any_sync(kFull, cur < end)) {
            bool want = false;
            int32_t v = 0;
            int64_t vb = 0;
            uint32_t vd = 0;
            if (cur < end) {
                v = __ldg(p.g.col + cur);
                const bool hit = SSSP ? sssp_relax(status, qcur, v, du, __ldg(p.g.w + cur), ctl)
                                      : bfs_claim(p.bitmap, status, v, level + 1);
                if (hit) {
                    vb = __ldg(p.g.off + v);
                    vd = (uint32_t)(__ldg(p.g.off + v + 1) - vb);
                    want = vd > 0;
                }
                ++cur;
            }
            wpush(wb, cnt, want, v, vb, vd);
            if (cnt > kWB - 32) wflush<OUTK, TILED>(wb, ws, cnt, o);
        }
    }
    __syncthreads();
    const uint32_t nbig = s_nbig < (uint32_t)kBigCap ? s_nbig : (uint32_t)kBigCap;
    for (uint32_t k = 0; k < nbig; ++k) {
        const int64_t i = s_big[k];
        const int64_t c0 = __ldg(in.beg + i);
        const int64_t n0 = __ldg(in.scan + i + 1) - __ldg(in.scan + i);
        const uint32_t d0 = SSSP ? sssp_source_dist(status, qcur, __ldg(in.v + i)) : 0u;
        // warp w takes the 32-edge stripes w, w + 8, w + 16, ... of the entry
        serve_range<SSSP, ITEMS, OUTK, TILED>(p, ctl, c0 + 32 * (int64_t)warp, c0 + n0, kBlock, d0, status, level,
                                              qcur, wb, ws, cnt, o);
    }
}

__device__ __forceinline__ void finish_hp_step(const StepParams &p, Ctl *ctl) {
    __threadfence();
    const unsigned long long pk = ld_volatile(&ctl->out_pack);
    const unsigned long long spk = ld_volatile(&ctl->sub_pack);
    int64_t sub_cnt = (int64_t)(spk >> 32);
    const int64_t sub_edges = (int64_t)(spk & 0xFFFFFFFFull);
    if (sub_cnt > p.list_cap) { ctl->error |= kErrCapacity; sub_cnt = p.list_cap; }
    const uint32_t kind = ctl->hp_kind;
    const int64_t step_edges = kind == 1u ? (int64_t)ctl->in_edges - sub_edges : (int64_t)ctl->in_edges;
    trace_append(ctl, kind == 1u ? kModeHpSub : (kind == 3u ? kModeHpBin : kModeHpWd), ctl->in_cnt, step_edges);
    ctl->relaxed += (unsigned long long)step_edges;
    ctl->step += 1;
    ctl->blocks_done = 0;
    const int64_t thr = p.hp_threshold;
    if (kind == 1u && sub_cnt > 0) {
        const uint32_t so = ctl->hp_from == kHpFromSuper ? 0u : (ctl->sub_in ^ 1u);
        const bool sub_next = !(thr > 0 && sub_cnt < thr);
        ctl->hp_lvl += 1;
        // a list within the first hp_depth of the chain gets its own MDT
        // (k_hp_mdt, before the next sub-iteration); later ones keep it
        if (p.hp_depth > 1 && ctl->hp_lvl < (uint32_t)p.hp_depth && sub_next) ctl->hp_mdt_pending = 1;
        p.subs[so].scan[sub_cnt] = (int32_t)sub_edges;
        ctl->hp_from = kHpFromSub;
        ctl->sub_in = so;
        ctl->in_cnt = (uint32_t)sub_cnt;
        ctl->in_edges = (uint64_t)sub_edges;
        ctl->sub_pack = 0ull;
        ctl->hp_sub += 1;
        ctl->hp_kind = (thr > 0 && sub_cnt < thr) ? 2u : 1u;
        set_loop(p, ctl, true);
    } else {
        int64_t cnt = (int64_t)(pk >> 32);
        const int64_t edges = (int64_t)(pk & 0xFFFFFFFFull);
        if (cnt > p.list_cap) { ctl->error |= kErrCapacity; cnt = p.list_cap; }
        const uint32_t out = ctl->par ^ 1u;
        p.lists[out].scan[cnt] = (int32_t)edges;
        ctl->par = out;
        ctl->in_cnt = (uint32_t)cnt;
        ctl->in_edges = (uint64_t)edges;
        ctl->out_pack = 0ull;
        ctl->sub_pack = 0ull;
        ctl->level += 1;
        ctl->hp_from = kHpFromSuper;
        ctl->hp_sub = 0;
        ctl->hp_mdt = (uint32_t)p.mdt;
        ctl->hp_lvl = 0;
        ctl->hp_mdt_pending = 0;
        ctl->sub_maxdeg = 0ull;
        ctl->hp_kind = (thr > 0 && cnt < thr) ? 2u : (p.hp_mode == 1 ? 3u : 1u);
        set_loop(p, ctl, cnt > 0);
    }
    __threadfence();
}

// ---------------------------------------------------------------------------
// Node splitting with the granules served at three granularities (ns_mode
// 1): the list holds the paper's granules (ceil(d / MDT) runs of at most MDT
// edges per split node, Sec. III-B), and each granule goes to a thread, a
// warp or the whole CTA by its length, as in the degree-binned HP step.
template <bool SSSP, int ITEMS>
__global__ void __launch_bounds__(kBlock) k_step_ns_binned(StepParams p) {
    __shared__ WarpBuf s_wb[kWarps];
    __shared__ WarpScratch s_ws[kWarps];
    Ctl *ctl = p.ctl;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    uint32_t *status = ctl->status;
    FlushOut o;
    o.list = p.lists[par ^ 1u];
    o.elist = nullptr;
    o.pack = &ctl->out_pack;
    o.cap = p.list_cap;
    o.tile_cap = p.tile_cap;
    o.tile = (int32_t)kTileGrain;
    o.mdt = p.mdt;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    o.child_first = nullptr;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t cnt = 0;
    binned_step<SSSP, ITEMS, kOutGranule, false>(p, ctl, p.lists[par], in_cnt, p.thread_max, status, level, qcur,
                                                 s_wb[warp], s_ws[warp], cnt, o);
    wflush<kOutGranule, false>(s_wb[warp], s_ws[warp], cnt, o);
    if (block_is_last(ctl) && threadIdx.x == 0) finish_plain_step(p, ctl, true, p.list_cap);
}

template <bool SSSP, int ITEMS>
__global__ void __launch_bounds__(kBlock) k_step_hp(StepParams p) {
    __shared__ WarpBuf s_wb[kWarps];   // updated nodes -> next super list
    __shared__ WarpBuf s_sb[kWarps];   // unfinished nodes -> next sub-list
    __shared__ WarpScratch s_ws[kWarps];
    Ctl *ctl = p.ctl;
    const uint32_t par = ctl->par;
    const int64_t in_cnt = ctl->in_cnt;
    const int64_t E = (int64_t)ctl->in_edges;
    const uint32_t level = ctl->level;
    uint32_t *const qcur = queued_half(p.bitmap, p.bm_words, level);
    if (SSSP) clear_next_queued(p.bitmap, p.bm_words, level);
    const uint32_t kind = ctl->hp_kind;
    const uint32_t from = ctl->hp_from;
    const uint32_t sub_in = ctl->sub_in;
    uint32_t *status = ctl->status;
    const NodeList in = from == kHpFromSuper ? p.lists[par] : p.subs[sub_in];
    FlushOut osup;
    osup.list = p.lists[par ^ 1u];
    osup.elist = nullptr;
    osup.pack = &ctl->out_pack;
    osup.cap = p.list_cap;
    osup.tile_cap = p.tile_cap;
    osup.tile = (int32_t)kTileGrain;
    osup.mdt = p.mdt;
    osup.err = &ctl->error;
    osup.pushes = &ctl->pushes;
    FlushOut osub = osup;
    osub.list = p.subs[from == kHpFromSuper ? 0u : (sub_in ^ 1u)];
    osub.pack = &ctl->sub_pack;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    WarpBuf &wb = s_wb[warp];
    WarpBuf &sb = s_sb[warp];
    WarpScratch &ws = s_ws[warp];
    uint32_t cnt = 0, scnt = 0;
    if (kind == 2u) {
        wd_walk<SSSP, ITEMS>(p, ctl, in, in_cnt, E, wb, ws, cnt, osup, status, level, qcur);
    } else if (kind == 3u) {
        // a thread serves at most min(MDT, thread_max) edges: on a skewed
        // graph the histogram MDT runs into the thousands
        const int64_t tmax = p.mdt < p.thread_max ? (int64_t)p.mdt : (int64_t)p.thread_max;
        binned_step<SSSP, ITEMS, kOutNode, true>(p, ctl, in, in_cnt, tmax, status, level, qcur, wb, ws, cnt, osup);
    } else {
        const int64_t mdt = (int64_t)ctl->hp_mdt;
        const bool track = p.hp_depth > 1;  // the sub-list's largest remaining degree, for k_hp_mdt
        const int64_t stride = (int64_t)gridDim.x * kBlock;
        for (int64_t base = (int64_t)blockIdx.x * kBlock + warp * 32; base < in_cnt; base += stride) {
            const int64_t i = base + lane;
            int64_t cur = 0, end = 0, rest = 0;
            uint32_t du = 0;
            int32_t u = 0;
            if (i < in_cnt) {
                cur = __ldg(in.beg + i);
                const int64_t len = __ldg(in.scan + i + 1) - __ldg(in.scan + i);
                if (cur < 0 || len < 0 || cur + len > p.g.m) {
                    atomicOr(&ctl->error, kErrBounds);
                    cur = 0;
                } else {
                    const int64_t take = len < mdt ? len : mdt;
                    end = cur + take;
                    rest = len - take;
                    u = __ldg(in.v + i);
                    if (SSSP) du = sssp_source_dist(status, qcur, u);
                }
            }
            // an entry skipped as redundant (SSSP, see sssp_source_dist) leaves no remainder
            const bool keep = rest > 0 && (!SSSP || du != kInf);
            if (track) {
                const uint32_t mx = __reduce_max_sync(kFull, keep ? (uint32_t)rest : 0u);
                if (lane == 0 && mx > 0) atomicMax(&ctl->sub_maxdeg, (unsigned long long)mx);
            }
            if (SSSP && du == kInf) end = cur;
            wpush(sb, scnt, keep, u, end, (uint32_t)rest);
            if (scnt > kWB - 32) wflush<kOutNode, true>(sb, ws, scnt, osub);
            while (__any_sync(kFull, cur < end)) {
                bool want = false;
                int32_t v = 0;
                int64_t vb = 0;
                uint32_t vd = 0;
                if (cur < end) {
                    v = __ldg(p.g.col + cur);
                    const bool hit = SSSP ? sssp_relax(status, qcur, v, du, __ldg(p.g.w + cur), ctl)
                                          : bfs_claim(p.bitmap, status, v, level + 1);
                    if (hit) {
                        vb = __ldg(p.g.off + v);
                        vd = (uint32_t)(__ldg(p.g.off + v + 1) - vb);
                        want = vd > 0;
                    }
                    ++cur;
                }
                wpush(wb, cnt, want, v, vb, vd);
                if (cnt > kWB - 32) wflush<kOutNode, true>(wb, ws, cnt, osup);
            }
        }
    }
    wflush<kOutNode, true>(wb, ws, cnt, osup);
    wflush<kOutNode, true>(sb, ws, scnt, osub);
    if (block_is_last(ctl) && threadIdx.x == 0) finish_hp_step(p, ctl);
}

}  // namespace lbk
