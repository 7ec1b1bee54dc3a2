// lb_bfs_wd_noalloc: BFS with the workload-decomposition kernel for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// entirely owned by another allocator (a framework's caching pool that has
// reserved the GPU), or a latency-bound service that must not allocate once
// it is running, because cudaMalloc can block and synchronise the device.
// This entry point takes the graph and the output buffer from the caller
// and keeps every other byte it needs (worklists, visited bitmap, loop
// state) in one fixed-size array of device memory declared in this file.
// Each GPU that loads the library holds that array until the process exits.
//
// Limits: n <= 131072 vertices and m <= 16777216 edges (about 3.6 MiB of
// scratch).  Every call on a device shares the array and finds the previous
// call's contents in it; the kernels reset what must start at zero (loop
// counters, the visited bitmap, the validation word and the output levels).
// The caller's CSR is checked on the device before any traversal (offsets
// start at 0, never decrease and end at m; every column is in [0, n)), so a
// malformed graph is refused instead of indexing outside the array.  Calls whose work
// overlaps on the GPU (different streams without ordering, or threads
// calling concurrently) race on the array and give wrong results.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lb_internal.cuh"

using namespace lbk;

namespace {

constexpr int64_t kNaMaxN = (int64_t)1 << 17;
constexpr int64_t kNaMaxM = (int64_t)1 << 24;
constexpr int32_t kNaTile = 2048;
constexpr int64_t kNaTiles = kNaMaxM / kTileGrain + 2;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the pieces inside the scratch array
constexpr size_t kOffCtl = 0;
constexpr size_t kOffBitmap = align256(kOffCtl + sizeof(Ctl));
constexpr int64_t kNaBitmapWords = ((kNaMaxN + 31) / 32 + 3) / 4 * 4;  // the BFS visited bits
constexpr size_t kListV = align256(sizeof(int32_t) * (size_t)kNaMaxN);
constexpr size_t kListBeg = align256(sizeof(int32_t) * (size_t)kNaMaxN);
constexpr size_t kListScan = align256(sizeof(int32_t) * (size_t)(kNaMaxN + 1));
constexpr size_t kListTiles = align256(sizeof(int32_t) * (size_t)kNaTiles);
constexpr size_t kListBytes = kListV + kListBeg + kListScan + kListTiles;
constexpr size_t kOffValid = align256(kOffBitmap + sizeof(uint32_t) * (size_t)kNaBitmapWords);
constexpr size_t kOffLists = align256(kOffValid + sizeof(uint32_t));
constexpr size_t kNaBytes = kOffLists + 2 * kListBytes;

static __device__ __align__(256) unsigned char lb_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
unsigned char *g_na_ptr[kMaxDevices] = {nullptr};


// Device address of the scratch array on the current device, looked up
// once per device with that device current.
cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, lb_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = (unsigned char *)p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

// Records the message lb_last_error() returns on this thread.
lb_status na_fail(lb_status s, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) snprintf(buf, sizeof(buf), "lb_bfs_wd_noalloc: %s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof(buf), "lb_bfs_wd_noalloc: %s", msg);
    set_last_error(buf);
    return s;
}

}  // namespace

extern "C" lb_status lb_bfs_wd_noalloc(const int64_t *offsets_dev, const int32_t *cols_dev, int64_t n, int64_t m,
                                       int32_t src, int32_t *levels_dev, void *stream) {
    set_last_error("");
    if (!offsets_dev || !levels_dev || (m > 0 && !cols_dev)) return na_fail(LB_ERR_ARG, "NULL pointer argument");
    if (n < 1 || n > kNaMaxN) return na_fail(LB_ERR_ARG, "n must be in [1, 131072] (the scratch array's limit)");
    if (m < 0 || m > kNaMaxM) return na_fail(LB_ERR_ARG, "m must be in [0, 16777216] (the scratch array's limit)");
    if (src < 0 || (int64_t)src >= n) return na_fail(LB_ERR_ARG, "source out of range");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return na_fail(LB_ERR_UNSUPPORTED, "device index too large");
    unsigned char *base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "cudaGetSymbolAddress", e);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "cudaDeviceGetAttribute", e);

    StepParams p;
    memset(&p, 0, sizeof(p));
    p.g = GraphDev{offsets_dev, cols_dev, nullptr, n, m};
    p.ctl = (Ctl *)(base + kOffCtl);
    p.bitmap = (uint32_t *)(base + kOffBitmap);
    p.bm_words = kNaBitmapWords;  // BFS reads only the first half: no second half is held
    for (int b = 0; b < 2; ++b) {
        unsigned char *L = base + kOffLists + (size_t)b * kListBytes;
        p.lists[b].v = (int32_t *)L;
        p.lists[b].beg = (int32_t *)(L + kListV);
        p.lists[b].scan = (int32_t *)(L + kListV + kListBeg);
        p.lists[b].tstart = (int32_t *)(L + kListV + kListBeg + kListScan);
    }
    p.list_cap = n;
    p.tile_cap = m / kTileGrain + 2;
    p.tile = kNaTile;
    p.mdt = 1;
    p.hp_threshold = 0;
    p.strategy = LB_WD;
    p.use_cond = 0;
    const int grid = step_blocks_per_sm(LB_WD, false, 0) * sms;
    cudaStream_t st = (cudaStream_t)stream;
    // the caller's CSR shape, checked before the traversal indexes with it
    uint32_t *verr = (uint32_t *)(base + kOffValid);
    uint32_t vword = 0;
    e = cudaMemsetAsync(verr, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_validate(p.g, verr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&vword, verr, sizeof(vword), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "CSR validation", e);
    if (vword & kErrShape)
        return na_fail(LB_ERR_ARG, "malformed CSR (offsets not 0..m and non-decreasing, or a column outside [0, n))");
    const uint32_t max_levels = (uint32_t)(n + 1);
    e = launch_prepare(p, src, (uint32_t *)levels_dev, LB_KIND_BFS, max_levels, (uint64_t)1 << 40,
                       (uint64_t)60 * 1000000000ull, st);
    if (e == cudaSuccess) e = launch_init(p, grid, st);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "launch", e);
    for (;;) {
        e = launch_step(LB_WD, false, p, grid, st);
        uint32_t active = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&active, &p.ctl->active, sizeof(active), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "worklist iteration", e);
        if (!active) break;
    }
    uint32_t err = 0;
    e = cudaMemcpyAsync(&err, &p.ctl->error, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(LB_ERR_CUDA, "reading the status word", e);
    if (err & (kErrCapacity | kErrShape | kErrBounds)) return na_fail(LB_ERR_INTERNAL, "device consistency check failed");
    if (err & (kErrIterCap | kErrDeadline)) return na_fail(LB_ERR_TIMEOUT, "iteration cap or time limit reached");
    return LB_OK;
}
