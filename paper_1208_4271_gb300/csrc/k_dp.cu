// k_dp.cu -- host dispatch of the blocked OptimizeXAxis DP kernel (k_dp.cuh)
// over its instances: precision x placement of the R table x level group.
// LEV, the levels kept in registers per pass, is fixed per launch: every
// launch covers row counts y whose tasks share one level group.
#include "k_dp.cuh"

namespace gm {

int dp_level_group(bool fp32, int nlev) {
  const int g = level_group(nlev);
  return fp32 ? g : (g > 20 ? 20 : g);
}

cudaError_t dp_configure(bool fp32, bool rsm, int lev, int smem, int threads, int* blocks_per_sm) {
  if (fp32) return rsm ? dp_f32_smem_configure(lev, smem, threads, blocks_per_sm)
                       : dp_f32_global_configure(lev, smem, threads, blocks_per_sm);
  return rsm ? dp_f64_smem_configure(lev, smem, threads, blocks_per_sm)
             : dp_f64_global_configure(lev, smem, threads, blocks_per_sm);
}

cudaError_t dp_launch(bool fp32, bool rsm, int lev, int grid, int threads, int smem,
                      cudaStream_t st, const DPParams& P, const DPPlan& S) {
  if (fp32) return rsm ? dp_f32_smem_launch(lev, grid, threads, smem, st, P, S)
                       : dp_f32_global_launch(lev, grid, threads, smem, st, P, S);
  return rsm ? dp_f64_smem_launch(lev, grid, threads, smem, st, P, S)
             : dp_f64_global_launch(lev, grid, threads, smem, st, P, S);
}

cudaError_t dp_occupancy_only(bool fp32, bool rsm, int lev, int smem, int threads, int* blocks_per_sm) {
  if (fp32) return rsm ? dp_f32_smem_occupancy(lev, smem, threads, blocks_per_sm)
                       : dp_f32_global_occupancy(lev, smem, threads, blocks_per_sm);
  return rsm ? dp_f64_smem_occupancy(lev, smem, threads, blocks_per_sm)
             : dp_f64_global_occupancy(lev, smem, threads, blocks_per_sm);
}

int dp_max_threads(bool fp32, bool rsm, int lev) {
  if (fp32) return rsm ? dp_f32_smem_max_threads(lev) : dp_f32_global_max_threads(lev);
  return rsm ? dp_f64_smem_max_threads(lev) : dp_f64_global_max_threads(lev);
}

}  // namespace gm
