// k_prep.cu -- per-variable and per-pair preparation kernels of libgmine:
// entropy tables, missing-sample counts, the tie-aware sort and rank, and
// EquipartitionYAxis of every (slot, row count).
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

// L(m) = m ln m (L(0) = 0), its float rounding, and ln m, for m = 0..n
// (Appendix items 9-10: entropies in nats from cell counts).
__global__ void k_tables(int n, double* L64, float* L32, double* lnt, int B, double c,
                         int64_t* rec_off) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= n;
       m += gridDim.x * blockDim.x) {
    const double lm = m > 0 ? log((double)m) : 0.0;
    const double L = m > 0 ? (double)m * lm : 0.0;
    L64[m] = L;
    L32[m] = (float)L;
    lnt[m] = lm;
  }
  // first int of the records of row count y within a (pair, orientation)
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y <= B / 2 + 1; y += gridDim.x * blockDim.x)
    rec_off[y] = y >= 2 ? rec_offset(B, n, c, y) : 0;
}

// Non-finite samples per variable (one warp per variable, coalesced rows).
__global__ void k_nonfinite(const double* __restrict__ vars, int64_t p, int n,
                            int32_t* nf) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (w >= p) return;
  const double* v = vars + w * (int64_t)n;
  int cnt = 0;
  for (int i = lane; i < n; i += 32) cnt += isfinite(v[i]) ? 0 : 1;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  if (lane == 0) nf[w] = cnt;
}

// Per pair of a chunk: its slots, n_used, B, and the list of pairs that need
// their own compacted ranks (a variable with a missing sample).
__global__ void k_pair_prep(const int32_t* __restrict__ pairs, int64_t pair0,
                            int64_t chunk, int64_t p, int n,
                            const int32_t* __restrict__ nf,
                            const int32_t* __restrict__ Btab, PairPrep pp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= chunk) return;
  const int32_t X = pairs[2 * (pair0 + i)];
  const int32_t Y = pairs[2 * (pair0 + i) + 1];
  pp.flags[i] = 0;
  if (X < 0 || Y < 0 || X >= p || Y >= p) {
    pp.slot[2 * i] = -1;
    pp.slot[2 * i + 1] = -1;
    pp.n_used[i] = 0;
    pp.B[i] = 0;
    pp.flags[i] = 1 << GMINE_E_ARG;
    return;
  }
  if (nf[X] == 0 && nf[Y] == 0) {
    pp.slot[2 * i] = X;
    pp.slot[2 * i + 1] = Y;
    pp.n_used[i] = n;
    pp.B[i] = Btab[n];
  } else {
    const int d = atomicAdd(pp.ndirty, 1);
    pp.dirty[d] = (int32_t)i;
    pp.slot[2 * i] = (int32_t)(p + 2 * d);
    pp.slot[2 * i + 1] = (int32_t)(p + 2 * d + 1);
    pp.n_used[i] = -1;  // filled in by the rank kernel
    pp.B[i] = -1;
  }
}

// ---------------------------------------------------------------------------
// Tie-aware sort and rank of one slot per CTA (bitonic sort of (key, sample)
// pairs in shared memory; the sample index breaks ties, so the order equals a
// stable argsort).  Outputs perm, pos, grp, gstart, ngroups, nslot.
//
// Clean slot s < p: variable s over all n samples (skipped when it has a
// missing sample).  Dirty slot s >= p: side (s - p) % 2 of dirty pair
// (s - p) / 2 of the chunk, over the samples where both of the pair's
// variables are finite (compacted, 0-based).
// ---------------------------------------------------------------------------
template <bool GLOBAL>
__global__ void __launch_bounds__(1024)
k_rank_t(const double* __restrict__ vars, int64_t p, int n,
       const int32_t* __restrict__ nf, const int32_t* __restrict__ pairs,
       int64_t pair0, PairPrep pp, const int32_t* __restrict__ Btab,
       int64_t slot_base, int64_t nslots, RankData rk, unsigned char* gscr,
       int64_t gscr_per_cta) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  int N2 = 1;
  while (N2 < n) N2 <<= 1;
  // keys and indices in shared memory, or (slots beyond the shared-memory
  // sort) in this CTA's global scratch; the scan buffer stays in shared
  unsigned char* kbase = GLOBAL ? gscr + (int64_t)blockIdx.x * gscr_per_cta : smem;
  uint64_t* key = reinterpret_cast<uint64_t*>(kbase);
  int* idx = reinterpret_cast<int*>(key + N2);
  int* tmp = GLOBAL ? reinterpret_cast<int*>(smem) : idx + N2;  // T + 1 ints
  for (int64_t sl = blockIdx.x; sl < nslots; sl += gridDim.x) {
  const int64_t slot = slot_base + sl;
  const double* xv = nullptr;
  const double* yv = nullptr;
  int side = 0;
  int64_t pair_local = -1;
  if (slot < p) {
    if (nf[slot] != 0) {
      if (tid == 0) {
        rk.nslot[slot] = 0;
        rk.ngroups[slot] = 0;
      }
      continue;
    }
    xv = vars + slot * (int64_t)n;
  } else {
    const int64_t d = (slot - p) / 2;
    if (d >= *pp.ndirty) continue;
    side = (int)((slot - p) % 2);
    pair_local = pp.dirty[d];
    const int32_t X = pairs[2 * (pair0 + pair_local)];
    const int32_t Y = pairs[2 * (pair0 + pair_local) + 1];
    xv = vars + (int64_t)X * n;
    yv = vars + (int64_t)Y * n;
  }
  __syncthreads();  // the previous slot's arrays are no longer read

  int m_used = n;
  if (slot < p) {
    for (int i = tid; i < N2; i += T) {
      key[i] = i < n ? order_key(xv[i]) : ~0ull;
      idx[i] = i;
    }
  } else {
    for (int i = tid; i < n; i += T) idx[i] = (isfinite(xv[i]) && isfinite(yv[i])) ? 1 : 0;
    __syncthreads();
    m_used = block_exclusive_scan(idx, n, tmp);
    for (int i = tid; i < n; i += T) {
      if (isfinite(xv[i]) && isfinite(yv[i])) key[idx[i]] = order_key(side ? yv[i] : xv[i]);
    }
    __syncthreads();
    for (int i = tid; i < N2; i += T) {
      if (i >= m_used) key[i] = ~0ull;
      idx[i] = i;
    }
    if (tid == 0 && side == 0) {
      pp.n_used[pair_local] = m_used;
      pp.B[pair_local] = Btab[m_used];
    }
  }
  __syncthreads();

  // bitonic sort ascending on (key, idx)
  for (int size = 2; size <= N2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < N2; i += T) {
        const int j = i ^ stride;
        if (j > i) {
          const uint64_t ki = key[i], kj = key[j];
          const int ii = idx[i], ij = idx[j];
          const bool gt = (ki > kj) || (ki == kj && ii > ij);
          const bool up = (i & size) == 0;
          if (gt == up) {
            key[i] = kj;
            key[j] = ki;
            idx[i] = ij;
            idx[j] = ii;
          }
        }
      }
      __syncthreads();
    }
  }

  int32_t* perm = rk.perm + slot * rk.stride;
  int32_t* pos = rk.pos + slot * rk.stride;
  int32_t* grp = rk.grp + slot * rk.stride;
  int32_t* gstart = rk.gstart + slot * (rk.stride + 1);
  // group-start flags into tmp-free storage: reuse the upper half of key as
  // int flags is unsafe (keys still read), so write flags into grp first.
  for (int m = tid; m < m_used; m += T) {
    perm[m] = idx[m];
    pos[idx[m]] = m;
  }
  __syncthreads();
  // flags in the idx array (perm already saved)
  for (int m = tid; m < m_used; m += T) idx[m] = (m == 0 || key[m] != key[m - 1]) ? 1 : 0;
  __syncthreads();
  for (int m = tid; m < m_used; m += T)
    if (idx[m]) key[m] = 1; else key[m] = 0;  // keep a copy of the flags
  __syncthreads();
  const int G = block_exclusive_scan(idx, m_used, tmp);
  for (int m = tid; m < m_used; m += T) {
    const int excl = idx[m];
    const bool start = key[m] != 0;
    grp[m] = start ? excl : excl - 1;
    if (start) gstart[excl] = m;
  }
  if (tid == 0) {
    gstart[G] = m_used;
    rk.ngroups[slot] = G;
    rk.nslot[slot] = m_used;
  }
  }  // slots
}

cudaError_t rank_launch(int grid, int threads, int smem, cudaStream_t st, const double* vars,
                        int64_t p, int n, const int32_t* nf, const int32_t* pairs, int64_t pair0,
                        PairPrep pp, const int32_t* Btab, int64_t slot_base, int64_t nslots,
                        RankData rk, unsigned char* gscr, int64_t gscr_per_cta) {
  auto k = gscr ? k_rank_t<true> : k_rank_t<false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (gscr)
    k_rank_t<true><<<grid, threads, smem, st>>>(vars, p, n, nf, pairs, pair0, pp, Btab, slot_base,
                                                nslots, rk, gscr, gscr_per_cta);
  else
    k_rank_t<false><<<grid, threads, smem, st>>>(vars, p, n, nf, pairs, pair0, pp, Btab, slot_base,
                                                 nslots, rk, gscr, gscr_per_cta);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// EquipartitionYAxis of every (slot, y): one thread per (slot, y), the row
// search of equipartition_bounds over the slot's tie groups.
// ---------------------------------------------------------------------------
__global__ void k_equi(int64_t slot_base, int64_t nslots, int64_t p,
                       const int32_t* __restrict__ Btab,
                       const int32_t* __restrict__ ndirty, RankData rk,
                       EquiData eq) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots * eq.R) return;
  const int64_t slot = slot_base + t / eq.R;
  if (slot >= p && (slot - p) / 2 >= *ndirty) return;
  const int y = 2 + (int)(t % eq.R);
  int32_t* bnd = eq.bounds + (slot * eq.R + (y - 2)) * eq.bstride;
  int32_t* yh = eq.yhat + slot * eq.R + (y - 2);
  const int m = rk.nslot[slot];
  const int B = m > 0 ? Btab[m] : 0;
  if (m < 4 || B < 4 || y > B / 2) {
    *yh = 0;
    return;
  }
  const int32_t* gs = rk.gstart + slot * (rk.stride + 1);
  const int32_t* grp = rk.grp + slot * rk.stride;
  *yh = equipartition_bounds(gs, grp, rk.ngroups[slot], m, y, bnd);
}

// EquipartitionYAxis of every clean variable into one given number of rows
// y (the single-step entry point): one thread per variable.
__global__ void k_equi_single(int64_t p, int y, RankData rk, EquiData eq) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= p) return;
  const int m = rk.nslot[v];
  int32_t* bnd = eq.bounds + v * eq.bstride;
  if (m < 1) {
    eq.yhat[v] = 0;
    return;
  }
  const int32_t* gs = rk.gstart + v * (rk.stride + 1);
  const int32_t* grp = rk.grp + v * rk.stride;
  eq.yhat[v] = equipartition_bounds(gs, grp, rk.ngroups[v], m, y, bnd);
}

}  // namespace gm
