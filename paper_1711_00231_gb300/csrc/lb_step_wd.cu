// WD (workload decomposition) step kernels and the persistent small-list
// kernel.
#include "lb_launch.h"
#include "lb_steps.cuh"

namespace lbk {

cudaError_t launch_step_wd(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
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
