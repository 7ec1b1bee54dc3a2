// BS (node per thread), NS (granule per thread, or binned granules) and
// physical-NS step kernels.
#include "lb_launch.h"
#include "lb_steps.cuh"

namespace lbk {

template <bool S, int K>
static int occ() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_entry<S, K>, kBlock, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_step_entry(bool sssp, bool granules, const StepParams &p, int grid, cudaStream_t st) {
    if (sssp) {
        if (granules) k_step_entry<true, kOutGranule><<<grid, kBlock, 0, st>>>(p);
        else k_step_entry<true, kOutNode><<<grid, kBlock, 0, st>>>(p);
    } else {
        if (granules) k_step_entry<false, kOutGranule><<<grid, kBlock, 0, st>>>(p);
        else k_step_entry<false, kOutNode><<<grid, kBlock, 0, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_ns_binned(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    if (sssp) k_step_ns_binned<true, kItemsWd><<<grid, kBlock, 0, st>>>(p);
    else k_step_ns_binned<false, kItemsWd><<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

int occupancy_step_ns_binned(bool sssp) {
    int nb = 0;
    cudaError_t e = sssp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_ns_binned<true, kItemsWd>, kBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_ns_binned<false, kItemsWd>, kBlock, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_step_phys(bool sssp, const StepParams &p, int grid, cudaStream_t st) {
    if (sssp) k_step_phys<true><<<grid, kBlock, 0, st>>>(p);
    else k_step_phys<false><<<grid, kBlock, 0, st>>>(p);
    return cudaGetLastError();
}

int occupancy_step_phys(bool sssp) {
    int nb = 0;
    cudaError_t e = sssp ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_phys<true>, kBlock, 0)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_phys<false>, kBlock, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int occupancy_step_entry(bool sssp, bool granules) {
    if (sssp) return granules ? occ<true, kOutGranule>() : occ<true, kOutNode>();
    return granules ? occ<false, kOutGranule>() : occ<false, kOutNode>();
}

}  // namespace lbk
