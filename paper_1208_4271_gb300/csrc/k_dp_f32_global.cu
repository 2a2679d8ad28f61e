// k_dp_f32_global.cu -- the blocked OptimizeXAxis DP kernel (k_dp.cuh) instantiated for
// FP32 values with the R table in global scratch, one instance per level group.
#include "k_dp.cuh"

namespace gm {

GM_DP_WRAPPERS(float, false, dp_f32_global, case 4: return k_dp<float, false, 4>; case 8: return k_dp<float, false, 8>; case 12: return k_dp<float, false, 12>; case 16: return k_dp<float, false, 16>; case 20: return k_dp<float, false, 20>; case 24: return k_dp<float, false, 24>; case 32: return k_dp<float, false, 32>; case 36: return k_dp<float, false, 36>; default: return k_dp<float, false, 40>;)

}  // namespace gm
