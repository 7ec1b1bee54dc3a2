// EP (edge-based, COO) step kernels, with and without work chunking.
#include "lb_launch.h"
#include "lb_steps.cuh"

namespace lbk {

template <bool S, bool C>
static int occ() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_ep<S, kItemsEp, C>, kBlock, 0) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_step_ep(bool sssp, bool chunk, const StepParams &p, int grid, cudaStream_t st) {
    if (sssp) {
        if (chunk) k_step_ep<true, kItemsEp, true><<<grid, kBlock, 0, st>>>(p);
        else k_step_ep<true, kItemsEp, false><<<grid, kBlock, 0, st>>>(p);
    } else {
        if (chunk) k_step_ep<false, kItemsEp, true><<<grid, kBlock, 0, st>>>(p);
        else k_step_ep<false, kItemsEp, false><<<grid, kBlock, 0, st>>>(p);
    }
    return cudaGetLastError();
}

int occupancy_step_ep(bool sssp, bool chunk) {
    if (sssp) return chunk ? occ<true, true>() : occ<true, false>();
    return chunk ? occ<false, true>() : occ<false, false>();
}

}  // namespace lbk
