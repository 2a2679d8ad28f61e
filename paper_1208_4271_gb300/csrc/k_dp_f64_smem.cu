// k_dp_f64_smem.cu -- the blocked OptimizeXAxis DP kernel (k_dp.cuh) instantiated for
// FP64 values with the R table in shared memory, one instance per level group.
#include "k_dp.cuh"

namespace gm {

GM_DP_WRAPPERS(double, true, dp_f64_smem, case 4: return k_dp<double, true, 4>; case 8: return k_dp<double, true, 8>; case 12: return k_dp<double, true, 12>; case 16: return k_dp<double, true, 16>; default: return k_dp<double, true, 20>;)

}  // namespace gm
