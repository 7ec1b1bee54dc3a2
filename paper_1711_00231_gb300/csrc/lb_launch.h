// Per-translation-unit launchers of the step kernels (one TU per strategy
// family so the kernels compile in parallel).
#pragma once

#include "lb_internal.cuh"

namespace lbk {

constexpr int kItemsWd = 4;  // edges per thread per round in WD tiles
constexpr int kItemsEp = 4;  // worklist edges per thread per round in EP

cudaError_t launch_step_entry(bool sssp, bool granules, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_entry(bool sssp, bool granules);
cudaError_t launch_step_wd(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_wd(bool sssp);
cudaError_t launch_step_ep(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_ep(bool sssp);
cudaError_t launch_step_hp(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_hp(bool sssp);

}  // namespace lbk
