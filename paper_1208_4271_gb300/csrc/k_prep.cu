// k_prep.cu -- per-variable and per-pair preparation kernels of libgmine:
// entropy tables, missing-sample counts, the tie-aware sort and rank, and
// EquipartitionYAxis of every (slot, row count).
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

// L(m) = m ln m (L(0) = 0), its float rounding, and ln m, for m = 0..n
// (Appendix items 9-10: entropies in nats from cell counts).
// nL < 0 skips the tables and writes only the record offsets of a batch of
// n samples and B = B(n).
__global__ void k_tables(int nL, double* L64, float* L32, double* lnt, int B, int n, double c,
                         int64_t* rec_off) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= nL;
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

// Samples used by every pair of a batch (both variables finite) and its B,
// one warp per pair: count[2 i] = n_used, count[2 i + 1] = B (0 and 0 for a
// pair index outside [0, p)).
__global__ void k_pair_count(const double* __restrict__ vars, int64_t p, int64_t n,
                             const int32_t* __restrict__ pairs, int64_t n_pairs,
                             const uint8_t* __restrict__ aidx, const int32_t* __restrict__ Btab,
                             int64_t btab_stride, int32_t* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= n_pairs) return;
  const int32_t X = pairs[2 * i], Y = pairs[2 * i + 1];
  if (X < 0 || Y < 0 || X >= p || Y >= p) {
    if (lane == 0) count[2 * i] = count[2 * i + 1] = 0;
    return;
  }
  const double* x = vars + (int64_t)X * n;
  const double* y = vars + (int64_t)Y * n;
  int m = 0;
  for (int64_t j = lane; j < n; j += 32) m += (isfinite(x[j]) && isfinite(y[j])) ? 1 : 0;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m += __shfl_xor_sync(0xffffffffu, m, d);
  if (lane == 0) {
    count[2 * i] = m;
    count[2 * i + 1] = Btab[(aidx ? (int64_t)aidx[i] * btab_stride : 0) + m];
  }
}

// Per pair of a chunk: its slots, n_used, B, and the list of pairs that need
// their own compacted ranks (a variable with a missing sample, or every pair
// when pp.all_dirty).  p validates the pair's indices.
__global__ void k_pair_prep(const int32_t* __restrict__ pairs, int64_t pair0,
                            int64_t chunk, int64_t p, int n,
                            const int32_t* __restrict__ nf,
                            const int32_t* __restrict__ Btab, PairPrep pp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= chunk) return;
  const int64_t pi = pair_index(pp, pair0 + i);
  const int32_t X = pairs[2 * pi];
  const int32_t Y = pairs[2 * pi + 1];
  pp.flags[i] = 0;
  if (X < 0 || Y < 0 || X >= p || Y >= p) {
    pp.slot[2 * i] = -1;
    pp.slot[2 * i + 1] = -1;
    pp.n_used[i] = 0;
    pp.B[i] = 0;
    pp.flags[i] = 1 << GMINE_E_ARG;
    return;
  }
  if (!pp.all_dirty && nf[X] == 0 && nf[Y] == 0) {
    pp.slot[2 * i] = X;
    pp.slot[2 * i + 1] = Y;
    pp.n_used[i] = n;
    pp.B[i] = btab_of(Btab, pp, pi)[n];
  } else {
    const int d = atomicAdd(pp.ndirty, 1);
    pp.dirty[d] = (int32_t)i;
    pp.slot[2 * i] = (int32_t)(pp.slot0 + 2 * d);
    pp.slot[2 * i + 1] = (int32_t)(pp.slot0 + 2 * d + 1);
    pp.n_used[i] = -1;  // filled in by the rank kernel
    pp.B[i] = -1;
  }
}

// ---------------------------------------------------------------------------
// Tie-aware sort and rank of one slot per CTA (bitonic sort of (key, sample)
// pairs in shared memory; the sample index breaks ties, so the order equals a
// stable argsort).  Outputs perm, pos, grp, gstart, ngroups, nslot.
//
// Clean slot s < pp.slot0: variable s over all n samples (skipped when it
// has a missing sample).  Dirty slot s >= pp.slot0: side (s - slot0) % 2 of
// dirty pair (s - slot0) / 2 of the chunk, over the samples where both of
// the pair's variables are finite (compacted, 0-based; at most n of them).
// Variables are rows of n_row samples.
// ---------------------------------------------------------------------------
template <bool GLOBAL>
__global__ void __launch_bounds__(1024)
k_rank_t(const double* __restrict__ vars, int64_t n_row, int n,
       const int32_t* __restrict__ nf, const int32_t* __restrict__ pairs,
       int64_t pair0, PairPrep pp, const int32_t* __restrict__ Btab,
       int64_t slot_base, int64_t nslots, RankData rk, unsigned char* gscr,
       int64_t gscr_per_cta) {
  const int64_t p = pp.slot0;
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
  int64_t pair_local = -1, pair_global = -1;
  if (slot < p) {
    if (nf[slot] != 0) {
      if (tid == 0) {
        rk.nslot[slot] = 0;
        rk.ngroups[slot] = 0;
      }
      continue;
    }
    xv = vars + slot * n_row;
  } else {
    const int64_t d = (slot - p) / 2;
    if (d >= *pp.ndirty) continue;
    side = (int)((slot - p) % 2);
    pair_local = pp.dirty[d];
    pair_global = pair_index(pp, pair0 + pair_local);
    const int32_t X = pairs[2 * pair_global];
    const int32_t Y = pairs[2 * pair_global + 1];
    xv = vars + (int64_t)X * n_row;
    yv = vars + (int64_t)Y * n_row;
  }
  __syncthreads();  // the previous slot's arrays are no longer read

  int m_used = n;
  if (slot < p) {
    for (int i = tid; i < N2; i += T) {
      key[i] = i < n ? order_key(xv[i]) : ~0ull;
      idx[i] = i;
    }
  } else {
    // compaction of the pair's finite samples, one tile of T samples of the
    // row at a time: warp ballots, then the warps' counts scanned by warp 0
    // (tmp[0..31] exclusive offsets, tmp[32] the tile's total)
    const int lane = tid & 31, w = tid >> 5;
    int run = 0;
    for (int64_t base = 0; base < n_row; base += T) {
      const int64_t i = base + tid;
      const bool f = i < n_row && isfinite(xv[i]) && isfinite(yv[i]);
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) tmp[w] = __popc(bal);
      __syncthreads();
      if (w == 0) {
        const int v = lane < (T >> 5) ? tmp[lane] : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += o;
        }
        tmp[lane] = incl - v;
        if (lane == 31) tmp[32] = incl;
      }
      __syncthreads();
      const int pos = run + tmp[w] + __popc(bal & ((1u << lane) - 1u));
      if (f && pos < N2) key[pos] = order_key(side ? yv[i] : xv[i]);
      run += tmp[32];
      __syncthreads();
    }
    m_used = min(run, n);
    for (int i = tid; i < N2; i += T) {
      if (i >= m_used) key[i] = ~0ull;
      idx[i] = i;
    }
    if (tid == 0 && side == 0) {
      pp.n_used[pair_local] = m_used;
      pp.B[pair_local] = btab_of(Btab, pp, pair_global)[m_used];
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
                        int64_t n_row, int n, const int32_t* nf, const int32_t* pairs, int64_t pair0,
                        PairPrep pp, const int32_t* Btab, int64_t slot_base, int64_t nslots,
                        RankData rk, unsigned char* gscr, int64_t gscr_per_cta) {
  auto k = gscr ? k_rank_t<true> : k_rank_t<false>;
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  if (gscr)
    k_rank_t<true><<<grid, threads, smem, st>>>(vars, n_row, n, nf, pairs, pair0, pp, Btab, slot_base,
                                                nslots, rk, gscr, gscr_per_cta);
  else
    k_rank_t<false><<<grid, threads, smem, st>>>(vars, n_row, n, nf, pairs, pair0, pp, Btab, slot_base,
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
