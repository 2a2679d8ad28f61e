// k_pearson.cu -- Pearson correlation of each listed pair and the
// non-linearity index MIC - rho^2: the linear statistics the paper reports
// beside the four MINE statistics (Fig. 1 caption; SI Sec. 2A).
//
// One warp per pair (grid-stride over the pairs).  Over the samples where
// both variables are finite (the pairs' NaN rule): the lanes sum the count
// and the two variables, the sums meet in a warp reduction, then a second
// pass sums the centred products and squares the same way (two passes: no
// cancellation from raw moments);
//   rho = S_xy / sqrt(S_xx * S_yy),
// NaN when fewer than two samples remain or a variance is zero.  The index
// is MIC - rho^2 for a pair whose MINE score is valid (status OK), NaN
// otherwise.  Double precision throughout; only the order of the additions
// differs from a sequential sum.
#include <cmath>

#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__global__ void __launch_bounds__(256) k_pearson(const double* __restrict__ vars, int64_t p, int64_t n,
                                                 const int32_t* __restrict__ pairs, int64_t n_pairs,
                                                 const gmine_pair_score* __restrict__ scores,
                                                 double* __restrict__ rho, double* __restrict__ nonlin) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  for (int64_t pr = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pr < n_pairs; pr += nw) {
    const int32_t iu = pairs[2 * pr], iv = pairs[2 * pr + 1];
    double r = qnan;
    if (iu >= 0 && iu < p && iv >= 0 && iv < p) {
      const double* __restrict__ x = vars + (int64_t)iu * n;
      const double* __restrict__ y = vars + (int64_t)iv * n;
      double sx = 0.0, sy = 0.0, cnt = 0.0;
      for (int64_t i = lane; i < n; i += 32) {
        const double a = x[i], b = y[i];
        if (isfinite(a) && isfinite(b)) {
          sx += a;
          sy += b;
          cnt += 1.0;
        }
      }
      sx = warp_sum(sx);
      sy = warp_sum(sy);
      cnt = warp_sum(cnt);
      if (cnt >= 2.0) {
        const double mx = sx / cnt, my = sy / cnt;
        double sxy = 0.0, sxx = 0.0, syy = 0.0;
        for (int64_t i = lane; i < n; i += 32) {
          const double a = x[i], b = y[i];
          if (isfinite(a) && isfinite(b)) {
            const double dx = a - mx, dy = b - my;
            sxy += dx * dy;
            sxx += dx * dx;
            syy += dy * dy;
          }
        }
        sxy = warp_sum(sxy);
        sxx = warp_sum(sxx);
        syy = warp_sum(syy);
        if (sxx > 0.0 && syy > 0.0) r = sxy / sqrt(sxx * syy);
      }
    }
    if (lane == 0) {
      rho[pr] = r;
      if (nonlin) {
        const bool ok = scores && scores[pr].status == GMINE_OK && r == r;
        nonlin[pr] = ok ? scores[pr].mic - r * r : qnan;
      }
    }
  }
}

}  // namespace

cudaError_t pearson_launch(int grid, cudaStream_t st, const double* d_vars, int64_t p, int64_t n,
                           const int32_t* d_pairs, int64_t n_pairs, const gmine_pair_score* d_scores,
                           double* d_rho, double* d_nonlin) {
  k_pearson<<<grid, 256, 0, st>>>(d_vars, p, n, d_pairs, n_pairs, d_scores, d_rho, d_nonlin);
  return cudaGetLastError();
}

}  // namespace gm
