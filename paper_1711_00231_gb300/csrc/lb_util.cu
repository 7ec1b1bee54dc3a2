// Query set-up and tear-down kernels, one-time preprocessing (COO build,
// MDT histogram, node-splitting counts, CSR validation), the parent-tree
// pass, the workload-decomposition offset inspector, and the step-kernel
// dispatcher.
#include "lb_launch.h"
#include "lb_device.cuh"

namespace lbk {

// ------------------------------------------------------------ dispatcher --

cudaError_t launch_step(int strategy, bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    switch (strategy) {
        case LB_BS: return launch_step_entry(sssp, false, p, grid, st);
        case LB_NS: return p.ns_mode == 1 ? launch_step_ns_binned(sssp, p, grid, st)
                                          : launch_step_entry(sssp, true, p, grid, st);
        case LB_NS_PHYS: return launch_step_phys(sssp, p, grid, st);
        case LB_WD: return launch_step_wd(sssp, p, grid, st);
        case LB_EP: return launch_step_ep(sssp, true, p, grid, st);
        case LB_EP_NOCHUNK: return launch_step_ep(sssp, false, p, grid, st);
        case LB_HP: return launch_step_hp(sssp, p, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

int step_blocks_per_sm(int strategy, bool sssp, int ns_mode) {
    switch (strategy) {
        case LB_BS: return occupancy_step_entry(sssp, false);
        case LB_NS: return ns_mode == 1 ? occupancy_step_ns_binned(sssp) : occupancy_step_entry(sssp, true);
        case LB_NS_PHYS: return occupancy_step_phys(sssp);
        case LB_WD: return occupancy_step_wd(sssp);
        case LB_EP: return occupancy_step_ep(sssp, true);
        case LB_EP_NOCHUNK: return occupancy_step_ep(sssp, false);
        case LB_HP: return occupancy_step_hp(sssp);
        default: return 1;
    }
}

// ------------------------------------------------------- query set-up --

// Worklist entries the source contributes (its node, its granules, or its
// edges) for the strategy's list kind.
__device__ __forceinline__ int64_t source_units(int strategy, int64_t deg, int32_t mdt) {
    if (deg == 0) return 0;
    if (strategy == LB_EP || strategy == LB_EP_NOCHUNK) return deg;
    if (strategy == LB_NS || strategy == LB_NS_PHYS) return deg <= mdt ? 1 : (deg + mdt - 1) / mdt;
    return 1;
}

__global__ void k_prepare(StepParams p, int32_t src, uint32_t *status, int kind, uint32_t max_levels,
                          uint64_t max_steps, uint64_t time_limit_ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctl *c = p.ctl;
    const int64_t deg = p.g.off[src + 1] - p.g.off[src];
    c->status = status;
    c->src = src;
    c->kind = kind;
    c->level = 0;
    c->par = 0;
    c->in_cnt = (uint32_t)source_units(p.strategy, deg, p.mdt);
    c->in_edges = (uint64_t)deg;
    c->out_pack = 0ull;
    c->sub_pack = 0ull;
    c->hp_from = kHpFromSuper;
    c->hp_sub = 0;
    c->sub_in = 0;
    c->hp_kind = (p.hp_threshold > 0 && (int64_t)c->in_cnt < p.hp_threshold) ? 2u : (p.hp_mode == 1 ? 3u : 1u);
    c->hp_mdt = (uint32_t)p.mdt;
    c->small_pack[0] = c->small_pack[1] = c->small_pack[2] = 0ull;
    c->bar_count = 0u;
    c->bar_stop = 0u;
    c->small_run = 0u;
    c->hp_lvl = 0;
    c->hp_mdt_pending = 0;
    c->sub_maxdeg = 0ull;
    c->blocks_done = 0;
    c->active = 1;
    c->error = 0;
    c->max_levels = max_levels;
    c->max_steps = max_steps;
    c->t_start = global_ns();
    c->t_deadline = c->t_start + time_limit_ns;
    c->step = 0;
    c->relaxed = 0ull;
    c->pushes = 0ull;
    c->trace_len = 0;
}

__global__ void k_init(StepParams p) {
    const Ctl *c = p.ctl;
    const int32_t src = c->src;
    const bool sssp = c->kind == 1;
    uint32_t *status = c->status;
    const int64_t n = p.g.n;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (((uintptr_t)status & 15u) == 0) {
        // 16-byte stores (the output buffer is usually 16-byte aligned)
        uint4 *s4 = reinterpret_cast<uint4 *>(status);
        const int64_t n4 = n / 4;
        for (int64_t i = tid; i < n4; i += stride) {
            uint4 x = make_uint4(kInf, kInf, kInf, kInf);
            if (i == src / 4) {
                const int32_t k = src % 4;
                if (k == 0) x.x = 0u;
                else if (k == 1) x.y = 0u;
                else if (k == 2) x.z = 0u;
                else x.w = 0u;
            }
            s4[i] = x;
        }
        for (int64_t i = 4 * n4 + tid; i < n; i += stride) status[i] = i == src ? 0u : kInf;
    } else {
        for (int64_t i = tid; i < n; i += stride) status[i] = i == src ? 0u : kInf;
    }
    if (!sssp) {
        // BFS: the visited bits (first half), the source already visited
        const int64_t words = (n + 31) / 32;
        for (int64_t wd = tid; wd < words; wd += stride)
            p.bitmap[wd] = wd == (src >> 5) ? (1u << (src & 31)) : 0u;
    } else {
        // SSSP: both queued halves start empty
        for (int64_t wd = tid; wd < 2 * p.bm_words; wd += stride) p.bitmap[wd] = 0u;
    }
    const int64_t beg = p.g.off[src];
    const int64_t deg = p.g.off[src + 1] - beg;
    if (p.strategy == LB_EP || p.strategy == LB_EP_NOCHUNK) {
        for (int64_t j = tid; j < deg; j += stride) p.elist[0][j] = (int32_t)(beg + j);
        return;
    }
    const NodeList L = p.lists[0];
    if (p.strategy == LB_NS_PHYS) {
        // every child distance starts unknown; the source's children start at 0
        const int32_t cf = p.child_first[src];
        const int64_t nk = deg > p.mdt ? (deg + p.mdt - 1) / p.mdt - 1 : 0;
        for (int64_t c = tid; c < p.n_children; c += stride) {
            const int64_t id = n + c;
            p.child_dist[c] = (cf >= 0 && id >= cf && id < cf + nk) ? 0u : kInf;
        }
    }
    if (p.strategy == LB_NS || p.strategy == LB_NS_PHYS) {
        const int64_t units = source_units(p.strategy, deg, p.mdt);
        const int32_t cf = p.strategy == LB_NS_PHYS ? p.child_first[src] : -1;
        for (int64_t j = tid; j < units; j += stride) {
            L.v[j] = (cf >= 0 && j > 0) ? cf + (int32_t)(j - 1) : src;
            L.beg[j] = (int32_t)(beg + j * p.mdt);
            L.scan[j] = (int32_t)(j * p.mdt);
        }
        if (tid == 0) L.scan[units] = (int32_t)deg;
        return;
    }
    if (tid == 0) {
        L.v[0] = src;
        L.beg[0] = (int32_t)beg;
        L.scan[0] = 0;
        L.scan[deg > 0 ? 1 : 0] = (int32_t)deg;
    }
    if (L.tstart != nullptr) {
        const int64_t tiles = (deg + kTileGrain - 1) / kTileGrain;
        for (int64_t k = tid; k < tiles && k < p.tile_cap; k += stride) L.tstart[k] = 0;
    }
}

// After the loop: an SSSP whose relaxations ever saturated reports overflow
// iff some final distance is still the saturated value.
__global__ void k_finish_query(StepParams p) {
    Ctl *c = p.ctl;
    if (!(c->error & kErrSaturated)) return;
    const uint32_t *status = c->status;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.g.n; i += stride)
        if (status[i] == kSat) {
            atomicOr(&c->error, kErrOverflow);
            return;
        }
}

// HP hierarchy depth > 1 (Sec. III-C: a large sub-worklist is partitioned
// again, the MDT deciding the split): before a sub-iteration whose input
// sub-list is still within the first hp_depth lists of the super-iteration's
// chain, that list gets its own MDT -- the histogram heuristic of Sec.
// III-B applied to the remaining degrees of its entries (bins of equal width
// over (0, maxRemaining], the tallest, smallest on a tie; MDT = max(1,
// floor(binIndex * maxRemaining / bins))).  A no-op launch otherwise.
__global__ void k_hp_mdt(StepParams p) {
    Ctl *c = p.ctl;
    if (!c->hp_mdt_pending) return;  // uniform
    const int bins = p.hist_bins;
    const int64_t maxd = (int64_t)c->sub_maxdeg;
    const int64_t cnt = c->in_cnt;
    const NodeList in = p.subs[c->sub_in];
    __shared__ uint32_t sh[kHistMax];
    for (int k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (maxd > 0)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
            const int64_t d = (int64_t)in.scan[i + 1] - in.scan[i];
            if (d <= 0 || d > maxd) continue;
            const int64_t k = (d * bins + maxd - 1) / maxd;  // 1-based bin
            atomicAdd(&sh[k - 1], 1u);
        }
    __syncthreads();
    for (int k = threadIdx.x; k < bins; k += blockDim.x)
        if (sh[k]) atomicAdd(&c->hp_hist[k], sh[k]);
    if (block_is_last(c) && threadIdx.x == 0) {
        __threadfence();
        int best = 0;
        for (int k = 1; k < bins; ++k)
            if (__ldcg(&c->hp_hist[k]) > __ldcg(&c->hp_hist[best])) best = k;
        const int64_t mdt = maxd > 0 ? ((int64_t)(best + 1) * maxd) / bins : 1;
        c->hp_mdt = (uint32_t)(mdt < 1 ? 1 : mdt);
        for (int k = 0; k < bins; ++k) c->hp_hist[k] = 0;
        c->sub_maxdeg = 0ull;
        c->hp_mdt_pending = 0;
        c->blocks_done = 0;
        __threadfence();
    }
}

cudaError_t launch_hp_mdt(const StepParams &p, int grid, cudaStream_t st) {
    k_hp_mdt<<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_prepare(const StepParams &p, int32_t src, uint32_t *status, int kind, uint32_t max_levels,
                           uint64_t max_steps, uint64_t time_limit_ns, cudaStream_t st) {
    k_prepare<<<1, 32, 0, st>>>(p, src, status, kind, max_levels, max_steps, time_limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_init(const StepParams &p, int grid, cudaStream_t st) {
    k_init<<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_finish_query(const StepParams &p, cudaStream_t st) {
    k_finish_query<<<256, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

// -------------------------------------------------- one-time preprocessing --

// COO source array (Sec. II-B: the edge-based method needs the source of
// every edge): a warp per node writes its id over its edge range.
__global__ void k_coo_build(GraphDev g, int32_t *coo_src) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const uint32_t lane = threadIdx.x & 31u;
    for (int64_t u = w0; u < g.n; u += warps) {
        const int64_t b = g.off[u], e = g.off[u + 1];
        for (int64_t j = b + lane; j < e; j += 32) coo_src[j] = (int32_t)u;
    }
}

cudaError_t launch_coo_build(const GraphDev &g, int32_t *coo_src, cudaStream_t st) {
    k_coo_build<<<1024, kBlock, 0, st>>>(g, coo_src);
    return cudaGetLastError();
}

// MDT histogram (Sec. III-B).  scratch[0] = max degree, scratch[1..bins] =
// bin heights.  result = {MDT, maxDeg, binIndex}.
__global__ void k_max_degree(GraphDev g, unsigned long long *scratch) {
    unsigned long long mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n; u += stride) {
        const unsigned long long d = (unsigned long long)(g.off[u + 1] - g.off[u]);
        mx = d > mx ? d : mx;
    }
    for (int k = 16; k > 0; k >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, mx, k);
        mx = o > mx ? o : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(&scratch[0], mx);
}

__global__ void k_degree_hist(GraphDev g, int32_t bins, unsigned long long *scratch) {
    extern __shared__ unsigned int sh[];
    for (int k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int64_t maxd = (int64_t)scratch[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (maxd > 0)
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n; u += stride) {
            const int64_t d = g.off[u + 1] - g.off[u];
            if (d == 0) continue;
            const int64_t k = (d * bins + maxd - 1) / maxd;  // 1-based bin: (k-1) max < d bins <= k max
            atomicAdd(&sh[k - 1], 1u);
        }
    __syncthreads();
    for (int k = threadIdx.x; k < bins; k += blockDim.x)
        if (sh[k]) atomicAdd(&scratch[1 + k], (unsigned long long)sh[k]);
}

__global__ void k_mdt_pick(int32_t bins, const unsigned long long *scratch, int64_t *result) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t maxd = (int64_t)scratch[0];
    if (maxd == 0) {
        result[0] = 0;
        result[1] = 0;
        result[2] = 0;
        return;
    }
    int32_t best = 1;
    for (int32_t k = 2; k <= bins; ++k)
        if (scratch[k] > scratch[best]) best = k;
    int64_t mdt = ((int64_t)best * maxd) / bins;
    result[0] = mdt < 1 ? 1 : mdt;
    result[1] = maxd;
    result[2] = best;
}

cudaError_t launch_mdt(const GraphDev &g, int32_t bins, unsigned long long *scratch, int64_t *result,
                       cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(bins + 1), st);
    if (e != cudaSuccess) return e;
    k_max_degree<<<608, kBlock, 0, st>>>(g, scratch);
    k_degree_hist<<<608, kBlock, sizeof(unsigned int) * (size_t)bins, st>>>(g, bins, scratch);
    k_mdt_pick<<<1, 32, 0, st>>>(bins, scratch, result);
    return cudaGetLastError();
}

// Child nodes node splitting creates at threshold mdt.
__global__ void k_ns_count(GraphDev g, int32_t mdt, unsigned long long *out) {
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < g.n; u += stride) {
        const int64_t d = g.off[u + 1] - g.off[u];
        if (d > mdt) s += (unsigned long long)((d + mdt - 1) / mdt - 1);
    }
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(kFull, s, k);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

cudaError_t launch_ns_count(const GraphDev &g, int32_t mdt, unsigned long long *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_ns_count<<<608, kBlock, 0, st>>>(g, mdt, out);
    return cudaGetLastError();
}

// Physical node split (Sec. III-B): child ids are handed out in node order.
// Block b of 1024 nodes first sums its children; a serial scan turns the
// block sums into offsets; then each block scans its nodes' child counts and
// writes child_first (n + offset, or -1) and parent_of for every child.
__device__ __forceinline__ int64_t ns_children_of(const GraphDev &g, int64_t u, int64_t mdt) {
    const int64_t d = g.off[u + 1] - g.off[u];
    return d > mdt ? (d + mdt - 1) / mdt - 1 : 0;
}

__global__ void k_ns_block_sums(GraphDev g, int32_t mdt, unsigned long long *sums) {
    __shared__ unsigned long long sh[32];
    const int64_t u = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    unsigned long long k = u < g.n ? (unsigned long long)ns_children_of(g, u, mdt) : 0ull;
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(kFull, k, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < 32; ++i) t += sh[i];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_ns_scan_sums(unsigned long long *sums, int64_t nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const unsigned long long x = sums[b];
        sums[b] = run;
        run += x;
    }
}

__global__ void k_ns_assign(GraphDev g, int32_t mdt, const unsigned long long *sums, int32_t *child_first,
                            int32_t *parent_of) {
    __shared__ unsigned long long warp_tot[32];
    const int64_t u = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned long long k = u < g.n ? (unsigned long long)ns_children_of(g, u, mdt) : 0ull;
    unsigned long long incl = k;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = warp_tot[lane];
        unsigned long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, wi, o);
            if ((int)lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    if (u >= g.n) return;
    const int64_t first = (int64_t)(sums[blockIdx.x] + warp_tot[wid] + incl - k);
    child_first[u] = k > 0 ? (int32_t)(g.n + first) : -1;
    for (unsigned long long j = 0; j < k; ++j) parent_of[first + (int64_t)j] = (int32_t)u;
}

cudaError_t launch_ns_phys_build(const GraphDev &g, int32_t mdt, int32_t *child_first, int32_t *parent_of,
                                 unsigned long long *block_sums, cudaStream_t st) {
    const int64_t nb = (g.n + 1023) / 1024;
    k_ns_block_sums<<<(unsigned)nb, 1024, 0, st>>>(g, mdt, block_sums);
    k_ns_scan_sums<<<1, 32, 0, st>>>(block_sums, nb);
    k_ns_assign<<<(unsigned)nb, 1024, 0, st>>>(g, mdt, block_sums, child_first, parent_of);
    return cudaGetLastError();
}

// CSR shape check for graphs created from device arrays.
__global__ void k_validate(GraphDev g, uint32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0 && (g.off[0] != 0 || g.off[g.n] != g.m)) atomicOr(err, kErrShape);
    for (int64_t u = tid; u < g.n; u += stride)
        if (g.off[u + 1] < g.off[u]) atomicOr(err, kErrShape);
    for (int64_t e = tid; e < g.m; e += stride) {
        const int32_t v = g.col[e];
        if (v < 0 || (int64_t)v >= g.n) atomicOr(err, kErrShape);
        if (g.w != nullptr && g.w[e] == 0u) atomicOr(err, kErrZeroWeight);
    }
}

cudaError_t launch_validate(const GraphDev &g, uint32_t *err, cudaStream_t st) {
    k_validate<<<1216, kBlock, 0, st>>>(g, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------ parents --

__global__ void k_parents_init(StepParams p, int32_t *parents) {
    const int32_t src = p.ctl->src;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.g.n; i += stride)
        parents[i] = i == src ? src : -1;
}

// Every reached u offers itself as parent of each out-neighbour v whose
// value it explains exactly (level[u] + 1, or min(dist[u] + w, saturated)).
// Any such u is a valid parent; with positive weights (and for BFS) the
// values strictly increase along parents, so the result is a tree.
template <bool SSSP>
__global__ void k_parents(StepParams p, int32_t *parents) {
    const uint32_t *status = p.ctl->status;
    const int32_t src = p.ctl->src;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const uint32_t lane = threadIdx.x & 31u;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; u < p.g.n; u += warps) {
        const uint32_t du = status[u];
        if (du == kInf) continue;
        const int64_t b = p.g.off[u], e = p.g.off[u + 1];
        for (int64_t j = b + lane; j < e; j += 32) {
            const int32_t v = p.g.col[j];
            if (v == src) continue;
            uint32_t want;
            if (SSSP) {
                const uint64_t a = (uint64_t)du + p.g.w[j];
                want = a >= kSat ? kSat : (uint32_t)a;
            } else {
                want = du + 1;
            }
            if (status[v] == want) parents[v] = (int32_t)u;
        }
    }
}

cudaError_t launch_parents(const StepParams &p, bool sssp, int32_t *parents, cudaStream_t st) {
    k_parents_init<<<608, kBlock, 0, st>>>(p, parents);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (sssp) k_parents<true><<<1216, kBlock, 0, st>>>(p, parents);
    else k_parents<false><<<1216, kBlock, 0, st>>>(p, parents);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

// ---------------------------------------------- WD offsets inspection --

// Pushes the F given entries, in order, through the production warp push
// buffer with tile = edgesPerThread = ceil(sum / T); the tile starts the
// flush writes are the per-thread NodeOffsets of Sec. III-A.
__global__ void k_wd_offsets(const int64_t *deg, int64_t F, int64_t T, NodeList list, Ctl *ctl, int64_t *ept_out) {
    __shared__ WarpBuf wb;
    __shared__ WarpScratch ws;
    const uint32_t lane = lane_id();
    int64_t E = 0;
    for (int64_t i = lane; i < F; i += 32) E += deg[i];
    for (int k = 16; k > 0; k >>= 1) E += __shfl_xor_sync(kFull, E, k);
    const int64_t ept = (E + T - 1) / T;
    if (lane == 0) *ept_out = ept;
    if (ept == 0) return;
    FlushOut o;
    o.list = list;
    o.elist = nullptr;
    o.pack = &ctl->out_pack;
    o.cap = F;
    o.tile_cap = T + 1;
    o.tile = (int32_t)ept;
    o.mdt = 1;
    o.err = &ctl->error;
    o.pushes = &ctl->pushes;
    uint32_t cnt = 0;
    for (int64_t c = 0; c < F; c += 32) {
        const int64_t i = c + lane;
        const bool want = i < F;
        wpush(wb, cnt, want, want ? (int32_t)i : 0, 0, want ? (uint32_t)deg[i] : 0u);
        if (cnt > kWB - 32) wflush<kOutNode, true>(wb, ws, cnt, o);
    }
    wflush<kOutNode, true>(wb, ws, cnt, o);
    if (lane == 0) list.scan[F] = (int32_t)E;
}

cudaError_t launch_wd_offsets(const int64_t *deg, int64_t F, int64_t T, NodeList list, Ctl *ctl, int64_t *ept_out,
                              cudaStream_t st) {
    k_wd_offsets<<<1, 32, 0, st>>>(deg, F, T, list, ctl, ept_out);
    return cudaGetLastError();
}

}  // namespace lbk
