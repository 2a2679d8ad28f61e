// kernels.h -- kernel declarations and the shared-memory plan of the task
// kernel, used by the libgmine host code.
#pragma once

#include <cstdint>

#include "gmine_internal.cuh"

namespace gm {

// Byte offsets of the task kernel's dynamic shared memory.  Region P (the
// per-task prologue arrays) is dead once the count table is built and is
// then overlaid by the DP tables (region W, offset 0) when they fit; region
// K (bounds, superclump ends, counts, entropy column, reductions) stays.
struct SmemPlan {
  int offP_Qs, offP_q, offP_mixed, offP_cflag, offP_grpU, offP_cgrp, offP_cstart;
  int sizeP;
  int w_bytes;  // DP tables in shared memory (0 if they live in scratch)
  int offK_eb, offK_scb, offK_cum, offK_Ecol, offK_V, offK_Varg, offK_tmp;
  int total;    // dynamic shared memory of one CTA
  int p_in_smem;           // 1: region P in shared memory, 0: in scratch
  int64_t scratch_P;       // bytes of region P in scratch (when not in smem)
  int64_t scratch_tables;  // global DP tables per CTA (when not in smem)
  int64_t scratch_A32;     // int argmax table per CTA (double path, trace)
  int64_t scratch_cuts;    // chosen-partition buffer per CTA
  int64_t scratch_total;
};

__global__ void k_tables(int n, double* L64, float* L32, double* lnt);
__global__ void k_nonfinite(const double* vars, int64_t p, int n, int32_t* nf);
__global__ void k_pair_prep(const int32_t* pairs, int64_t pair0, int64_t chunk,
                            int64_t p, int n, const int32_t* nf,
                            const int32_t* Btab, PairPrep pp);
__global__ void k_rank(const double* vars, int64_t p, int n, const int32_t* nf,
                       const int32_t* pairs, int64_t pair0, PairPrep pp,
                       const int32_t* Btab, int64_t slot_base, RankData rk);
__global__ void k_equi(int64_t slot_base, int64_t nslots, int64_t p,
                       const int32_t* Btab, const int32_t* ndirty, RankData rk,
                       EquiData eq);
cudaError_t task_configure(bool fp32, int smem, int threads, int* blocks_per_sm);
cudaError_t task_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                        const TaskParams& P, const SmemPlan& S);
__global__ void k_final(FinalParams F);
__global__ void k_equi_single(int64_t p, int y, RankData rk, EquiData eq);
__global__ void k_rank_export(RankData rk, int64_t p, int32_t* rank_out,
                              int32_t* perm_out, int32_t* groups_out);
__global__ void k_equi_export(RankData rk, EquiData eq, int64_t p, int y,
                              int32_t* Q_out, int32_t* yhat_out);

}  // namespace gm
