// k_final.cu -- per pair: M(x,y) = max(M_0(x,y), M_1(y,x)) over x*y <= B
// (Appendix items 1 and 4) and the four statistics (Sec. 1; Appendix items
// 1-2): MIC = max M, MAS = max |M(x,y) - M(y,x)|, MEV = max M over x = 2 or
// y = 2, MCN = min log2(xy) over the cells with M = MIC.  One warp per pair.
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

__device__ __forceinline__ int cell_of(int B, int x, int y) { return row_offset(B, y) + x - 2; }

__global__ void k_final(FinalParams F) {
  const int lane = threadIdx.x & 31;
  const int64_t pl = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (pl >= F.chunk_pairs) return;
  const int n = F.pp.n_used[pl];
  const int B = F.pp.B[pl];
  const int64_t pi = pair_index(F.pp, F.pair0 + pl);  // the pair's index in the batch
  gmine_pair_score sc;
  sc.mic = sc.mas = sc.mev = sc.mcn = 0.0;
  sc.m_offset = pi * F.m_stride;
  sc.n_used = n < 0 ? 0 : n;
  sc.B = B < 0 ? 0 : B;
  sc.m_cells = 0;
  sc.mcn_xy = 0;
  const int sx = F.pp.slot[2 * pl], sy = F.pp.slot[2 * pl + 1];
  const bool has_rows = n >= 4 && B >= 4 && sx >= 0 && sy >= 0;
  sc.yhat_x = has_rows ? F.eq_yhat[(int64_t)sx * F.R] : 0;
  sc.yhat_y = has_rows ? F.eq_yhat[(int64_t)sy * F.R] : 0;
  sc.reserved = 0;
  const int flags = F.pp.flags[pl];
  if ((flags & (1 << GMINE_E_ARG)) || n < 4 || B < 4) {
    sc.status = (flags & (1 << GMINE_E_ARG)) ? GMINE_E_ARG : GMINE_E_TOO_FEW;
    if (lane == 0) F.scores[pi] = sc;
    return;
  }
  const double* M0 = F.Mo + (pl * 2 + 0) * F.cells_max;
  const double* M1 = F.Mo + (pl * 2 + 1) * F.cells_max;
  double* Mout = F.M ? F.M + pi * F.m_stride : nullptr;
  int cells = 0;
  for (int y = 2; y <= B / 2; ++y) cells += B / y - 1;

  // pass 1: M, MIC, MEV
  double mic = -1.0, mev = -1.0;
  int c0 = 0;
  for (int y = 2; y <= B / 2; ++y) {
    const int nx = B / y - 1;
    for (int j = lane; j < nx; j += 32) {
      const int x = j + 2;
      const double a = M0[c0 + j];
      const double b = M1[cell_of(B, y, x)];
      const double m = a > b ? a : b;
      if (Mout) Mout[c0 + j] = m;
      mic = m > mic ? m : mic;
      if (x == 2 || y == 2) mev = m > mev ? m : mev;
    }
    c0 += nx;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    mic = fmax(mic, __shfl_xor_sync(0xffffffffu, mic, d));
    mev = fmax(mev, __shfl_xor_sync(0xffffffffu, mev, d));
  }
  // pass 2: MAS and MCN need MIC and both (x,y) and (y,x)
  double mas = 0.0;
  int mcn_xy = 0x7fffffff;
  c0 = 0;
  for (int y = 2; y <= B / 2; ++y) {
    const int nx = B / y - 1;
    for (int j = lane; j < nx; j += 32) {
      const int x = j + 2;
      const double a = M0[c0 + j];
      const double b = M1[cell_of(B, y, x)];
      const double m = a > b ? a : b;
      const double at = M0[cell_of(B, y, x)];
      const double bt = M1[c0 + j];
      const double mt = at > bt ? at : bt;
      const double dd = fabs(m - mt);
      mas = dd > mas ? dd : mas;
      if (m >= mic && x * y < mcn_xy) mcn_xy = x * y;
    }
    c0 += nx;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    mas = fmax(mas, __shfl_xor_sync(0xffffffffu, mas, d));
    mcn_xy = min(mcn_xy, __shfl_xor_sync(0xffffffffu, mcn_xy, d));
  }
  sc.mic = mic;
  sc.mas = mas;
  sc.mev = mev;
  sc.mcn = log2((double)mcn_xy);
  sc.mcn_xy = mcn_xy;
  sc.m_cells = cells;
  sc.status = (flags & (1 << GMINE_E_TIMEOUT))    ? GMINE_E_TIMEOUT
              : (flags & (1 << GMINE_E_CONSTANT)) ? GMINE_E_CONSTANT
                                                  : GMINE_OK;
  if (lane == 0) F.scores[pi] = sc;
}

// Exports for the single-step entry points.
__global__ void k_rank_export(RankData rk, int64_t p, int32_t* rank_out,
                              int32_t* perm_out, int32_t* groups_out) {
  const int64_t v = blockIdx.y;
  if (v >= p) return;
  const int n = rk.nslot[v];
  const int32_t* perm = rk.perm + v * rk.stride;
  const int32_t* grp = rk.grp + v * rk.stride;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    perm_out[v * rk.stride + m] = perm[m];
    rank_out[v * rk.stride + perm[m]] = grp[m];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) groups_out[v] = rk.ngroups[v];
}

__global__ void k_equi_export(RankData rk, EquiData eq, int64_t p, int y,
                              int32_t* Q_out, int32_t* yhat_out) {
  const int64_t v = blockIdx.y;
  if (v >= p) return;
  const int n = rk.nslot[v];
  const int yh = eq.yhat[v * eq.R + (y - 2)];
  const int32_t* bnd = eq.bounds + (v * eq.R + (y - 2)) * eq.bstride;
  const int32_t* perm = rk.perm + v * rk.stride;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    int lo = 0, hi = yh;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (bnd[mid] <= m) lo = mid; else hi = mid;
    }
    Q_out[v * rk.stride + perm[m]] = lo;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) yhat_out[v] = yh;
}

}  // namespace gm
