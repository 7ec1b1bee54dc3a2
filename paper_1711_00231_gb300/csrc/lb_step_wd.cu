// WD (workload decomposition) step kernels.
#include "lb_launch.h"
#include "lb_steps.cuh"

namespace lbk {

cudaError_t launch_step_wd(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    if (sssp) k_step_wd<true, kItemsWd><<<grid, kBlock, 0, st>>>(p);
    else k_step_wd<false, kItemsWdBfs><<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

int occupancy_step_wd(bool sssp) {
    int nb = 0;
    cudaError_t e = sssp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_wd<true, kItemsWd>, kBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_wd<false, kItemsWdBfs>, kBlock, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

}  // namespace lbk
