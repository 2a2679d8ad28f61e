// kernels.h -- kernel declarations and host-side launch wrappers used by the
// libgmine host code.
#pragma once

#include <cstdint>

#include "gmine_internal.cuh"

namespace gm {

__global__ void k_tables(int nL, double* L64, float* L32, double* lnt, int B, int n, double c,
                         int64_t* rec_off);
__global__ void k_pair_count(const double* vars, int64_t p, int64_t n, const int32_t* pairs,
                             int64_t n_pairs, const uint8_t* aidx, const int32_t* Btab,
                             int64_t btab_stride, int32_t* count);
__global__ void k_nonfinite(const double* vars, int64_t p, int n, int32_t* nf);
__global__ void k_pair_prep(const int32_t* pairs, int64_t pair0, int64_t chunk,
                            int64_t p, int n, const int32_t* nf,
                            const int32_t* Btab, PairPrep pp);
cudaError_t rank_launch(int grid, int threads, int smem, cudaStream_t st, const double* vars,
                        int64_t n_row, int n, const int32_t* nf, const int32_t* pairs, int64_t pair0,
                        PairPrep pp, const int32_t* Btab, int64_t slot_base, int64_t nslots,
                        RankData rk, unsigned char* gscr, int64_t gscr_per_cta);
__global__ void k_equi(int64_t slot_base, int64_t nslots, int64_t p,
                       const int32_t* Btab, const int32_t* ndirty, RankData rk,
                       EquiData eq);
__global__ void k_equi_single(int64_t p, int y, RankData rk, EquiData eq);
cudaError_t partition_configure(bool global, bool wide, int smem, int threads, int* blocks_per_sm);
cudaError_t partition_launch(bool global, bool wide, int grid, int threads, int smem,
                             cudaStream_t st, const PartParams& P);
__global__ void k_final(FinalParams F);
__global__ void k_rank_export(RankData rk, int64_t p, int32_t* rank_out,
                              int32_t* perm_out, int32_t* groups_out);
__global__ void k_equi_export(RankData rk, EquiData eq, int64_t p, int y,
                              int32_t* Q_out, int32_t* yhat_out);

// each DP kernel template is instantiated and launched in its own unit
int dp_level_group(bool fp32, int nlev);
cudaError_t dp_small_configure(bool fp32, int smem, int threads, int* blocks_per_sm);
cudaError_t dp_small_occupancy(bool fp32, int smem, int threads, int* blocks_per_sm);
cudaError_t dp_small_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                            const DPParams& P, const SmallPlan& S);
cudaError_t dp_configure(bool fp32, bool rsm, int lev, int smem, int threads, int* blocks_per_sm);
cudaError_t dp_launch(bool fp32, bool rsm, int lev, int grid, int threads, int smem,
                      cudaStream_t st, const DPParams& P, const DPPlan& S);
int dp_max_threads(bool fp32, bool rsm, int lev);  // the instance's launch bound
// blocks per SM at `smem` bytes, leaving the instance's attribute as it is
cudaError_t dp_occupancy_only(bool fp32, bool rsm, int lev, int smem, int threads, int* blocks_per_sm);
// one pair per instance set (k_dp_{f32,f64}_{smem,global}.cu); dp_configure
// and dp_launch dispatch to them
#define GM_DP_DECLARE(NAME)                                                            \
  cudaError_t NAME##_configure(int lev, int smem, int threads, int* blocks_per_sm);     \
  cudaError_t NAME##_launch(int lev, int grid, int threads, int smem, cudaStream_t st,  \
                            const DPParams& P, const DPPlan& S);                        \
  cudaError_t NAME##_occupancy(int lev, int smem, int threads, int* blocks_per_sm);     \
  int NAME##_max_threads(int lev);
GM_DP_DECLARE(dp_f32_smem)
GM_DP_DECLARE(dp_f32_global)
GM_DP_DECLARE(dp_f64_smem)
GM_DP_DECLARE(dp_f64_global)
#undef GM_DP_DECLARE

cudaError_t dp_two_configure(bool fp32, int smem, int threads, int* blocks_per_sm);
cudaError_t dp_two_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                          const DPParams& P, int off_rec, int rec_bytes);
// warp-per-task blocked DP (float path): lev levels in registers, tdw ints
// of the lane's superclump row in registers (8: yhat <= 7, 16: yhat <= 15)
bool dp_warp_supported(int lev, int tdw);
cudaError_t dp_warp_configure(int lev, int tdw, int smem, int threads, int* blocks_per_sm, bool set_attr);
cudaError_t dp_warp_launch(int lev, int tdw, int grid, int threads, int smem, cudaStream_t st,
                           const DPParams& P, const WarpPlan& S);
cudaError_t dp_mid_configure(bool fp32, int smem, int threads, int* blocks_per_sm, bool set_attr);
cudaError_t dp_mid_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                          const DPParams& P, const MidPlan& S);

// Pearson rho and the non-linearity index per pair (k_pearson.cu)
cudaError_t pearson_launch(int grid, cudaStream_t st, const double* d_vars, int64_t p, int64_t n,
                           const int32_t* d_pairs, int64_t n_pairs, const gmine_pair_score* d_scores,
                           double* d_rho, double* d_nonlin);

// Records a CUDA error for gmine_strerror (host code outside gmine_api.cu).
void note_cuda_error(cudaError_t e);

// Lets `func` launch with `smem` bytes of dynamic shared memory on the
// current device.  The attribute only ever grows (a high-water mark per
// kernel and device, under a lock): a call planning a smaller launch never
// lowers the limit another host thread's planned launch relies on.
cudaError_t allow_dynamic_smem(const void* func, int smem);

}  // namespace gm
