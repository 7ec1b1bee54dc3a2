// WD (workload decomposition) step kernels and the persistent small-list
// kernel.
#include "lb_launch.h"
#include "lb_steps.cuh"

namespace lbk {

// Preferred shared-memory carve-out of the WD step kernels in percent of
// the largest (-1: the driver's choice).  The rest of the unified L1 /
// shared memory caches the randomly read visited bitmap (BFS) and
// distances (SSSP).  25% selects the 64 KB configuration, which holds the
// resident CTAs' push buffers (BFS: 6 x (9.1 + 1) KB with 96-entry buffers;
// SSSP: 4 x (12.1 + 1) KB) and leaves 192 KB of L1; the driver's own choice
// left less.  Measured on R-MAT scale 24: BFS 1.764 -> 1.672 ms, SSSP 6.48
// -> 6.28 ms per query.
#ifndef LB_WD_CARVEOUT_BFS
#define LB_WD_CARVEOUT_BFS 25
#endif
#ifndef LB_WD_CARVEOUT_SSSP
#define LB_WD_CARVEOUT_SSSP 25
#endif

cudaError_t launch_step_wd(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    if (LB_WD_CARVEOUT_BFS >= 0 && !sssp) {
        cudaError_t e = cudaFuncSetAttribute(k_step_wd<false, kItemsWdBfs>,
                                             cudaFuncAttributePreferredSharedMemoryCarveout, LB_WD_CARVEOUT_BFS);
        if (e != cudaSuccess) return e;
    }
    if (LB_WD_CARVEOUT_SSSP >= 0 && sssp) {
        cudaError_t e = cudaFuncSetAttribute(k_step_wd<true, kItemsWdSssp>,
                                             cudaFuncAttributePreferredSharedMemoryCarveout, LB_WD_CARVEOUT_SSSP);
        if (e != cudaSuccess) return e;
    }
    if (sssp) k_step_wd<true, kItemsWdSssp><<<grid, kBlock, 0, st>>>(p);
    else k_step_wd<false, kItemsWdBfs><<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_small_levels(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    // cooperative: the kernel's CTAs wait on one another at a grid barrier,
    // so all of them must be resident at once
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sssp) return cudaLaunchKernelEx(&cfg, k_small_levels<true, kItemsWd>, p);
    return cudaLaunchKernelEx(&cfg, k_small_levels<false, kItemsWdBfs>, p);
}

int small_ctas_per_sm() { return LB_SMALL_CTAS; }

int occupancy_step_wd(bool sssp) {
    int nb = 0;
    cudaError_t e = sssp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_wd<true, kItemsWdSssp>, kBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_wd<false, kItemsWdBfs>, kBlock, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace lbk
