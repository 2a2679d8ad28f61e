// k_dp_f32_smem.cu -- the blocked OptimizeXAxis DP kernel (k_dp.cuh) instantiated for
// FP32 values with the R table in shared memory, one instance per level group.
#include "k_dp.cuh"

namespace gm {

GM_DP_WRAPPERS(float, true, dp_f32_smem, case 4: return k_dp<float, true, 4>; case 8: return k_dp<float, true, 8>; case 12: return k_dp<float, true, 12>; case 16: return k_dp<float, true, 16>; case 20: return k_dp<float, true, 20>; case 24: return k_dp<float, true, 24>; case 32: return k_dp<float, true, 32>; case 36: return k_dp<float, true, 36>; default: return k_dp<float, true, 40>;)

}  // namespace gm
