// Per-translation-unit launchers of the step kernels (one TU per strategy
// family so the kernels compile in parallel).
#pragma once

#include "lb_internal.cuh"

namespace lbk {

#ifndef LB_WD_ITEMS
#define LB_WD_ITEMS 3
#endif
#ifndef LB_EP_ITEMS
#define LB_EP_ITEMS 4
#endif
constexpr int kItemsWd = LB_WD_ITEMS;  // edges per thread per round in WD tiles
// BFS relax: 3 edges per thread per round (2.5% faster than 2 at R-MAT
// scale 24; its 32-bit walk leaves the registers for it)
#ifndef LB_WD_ITEMS_BFS
#define LB_WD_ITEMS_BFS 3
#endif
constexpr int kItemsWdBfs = LB_WD_ITEMS_BFS;
// SSSP WD step: 4 edges per thread per round at 4 CTAs per SM (64
// registers, no spills); 2% faster than 3 edges at 5 CTAs at R-MAT scale 24
#ifndef LB_WD_ITEMS_SSSP
#define LB_WD_ITEMS_SSSP 4
#endif
constexpr int kItemsWdSssp = LB_WD_ITEMS_SSSP;
constexpr int kItemsEp = LB_EP_ITEMS;  // worklist edges per thread per round in EP

cudaError_t launch_step_entry(bool sssp, bool granules, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_entry(bool sssp, bool granules);
cudaError_t launch_step_ns_binned(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_ns_binned(bool sssp);
cudaError_t launch_step_phys(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_phys(bool sssp);
cudaError_t launch_step_wd(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_wd(bool sssp);
cudaError_t launch_step_ep(bool sssp, bool chunk, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_ep(bool sssp, bool chunk);
cudaError_t launch_step_hp(bool sssp, const StepParams &p, int grid, cudaStream_t st);
int occupancy_step_hp(bool sssp);

}  // namespace lbk
