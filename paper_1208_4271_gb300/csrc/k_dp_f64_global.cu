// k_dp_f64_global.cu -- the blocked OptimizeXAxis DP kernel (k_dp.cuh) instantiated for
// FP64 values with the R table in global scratch, one instance per level group.
#include "k_dp.cuh"

namespace gm {

GM_DP_WRAPPERS(double, false, dp_f64_global, case 4: return k_dp<double, false, 4>; case 8: return k_dp<double, false, 8>; case 12: return k_dp<double, false, 12>; case 16: return k_dp<double, false, 16>; default: return k_dp<double, false, 20>;)

}  // namespace gm
