// gmine_internal.cuh -- device-side building blocks shared by the libgmine
// kernels (never by the CPU oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gmine.h"

namespace gm {

constexpr int kWarp = 32;
constexpr int kMaxRankN = 16384;  // largest slot sorted in shared memory
constexpr int kMaxN = 131072;     // largest n (the global-memory sort's scratch per CTA)
constexpr int kMaxN16 = 65535;    // positions and counts fit 16 bits up to here

// ---------------------------------------------------------------------------
// Ordering key of a double: unsigned integers compare like the doubles, -0.0
// and +0.0 get the same key (they are equal values, hence one tie group).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t order_key(double v) {
  if (v == 0.0) v = 0.0;
  uint64_t b = static_cast<uint64_t>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of `n` int flags/counts held in shared memory
// (in place).  Each thread scans a contiguous chunk; chunk totals are scanned
// by warp 0.  `tmp` needs blockDim.x + 1 ints.  Returns the total.  All
// threads of the block must call it.
// ---------------------------------------------------------------------------
__device__ inline int block_exclusive_scan(int* a, int n, int* tmp) {
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int per = (n + T - 1) / T;
  const int lo = min(n, tid * per);
  const int hi = min(n, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += a[i];
  tmp[tid] = s;
  __syncthreads();
  if (tid < kWarp) {
    // warp 0 scans the T chunk totals, 32 at a time
    int carry = 0;
    for (int base = 0; base < T; base += kWarp) {
      int v = (base + tid < T) ? tmp[base + tid] : 0;
      int incl = v;
#pragma unroll
      for (int d = 1; d < kWarp; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (tid >= d) incl += o;
      }
      if (base + tid < T) tmp[base + tid] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, kWarp - 1);
    }
    if (tid == 0) tmp[T] = carry;
  }
  __syncthreads();
  int run = tmp[tid];
  for (int i = lo; i < hi; ++i) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
  const int total = tmp[T];
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------------------
// EquipartitionYAxis over tie groups (SOM Alg. 3; Appendix items 3-4).
//
// The n points are in sorted order; tie group g covers sorted positions
// [gs[g], gs[g+1]) (gs[0] = 0, gs[G] = n) and grp[m] is the group of
// position m.  With the current row starting at position R0 (1-based index
// i = R0 + 1) and being row number `row` (1-based) of Y, the desired size is
// d = (n - R0) / (Y - row + 1); group S, starting at position P_S with |S|
// points, opens a new row iff '#' = P_S - R0 != 0 and
// |# + |S| - d| >= |# - d|, i.e. iff 2# + |S| >= 2d, i.e. iff
//     (P_S + P_S+|S| - 2 R0) * (Y - row + 1) >= 2 (n - R0)
// in exact integers.  The left side grows strictly with the group, so the
// first such group is found directly: with Tp = 2 R0 + ceil(2 (n - R0) /
// (Y - row + 1)) and p* = floor((Tp - 1) / 2), no group before grp[p*]
// qualifies and every group after it does.  So the next row starts at
// group grp[p*] if that group qualifies, else at grp[p*] + 1 (never before
// the second group of the row).
//
// Writes the row starts bounds[0..yhat] (bounds[yhat] = n) and returns yhat.
// Works on shared or global arrays (generic pointers).
// ---------------------------------------------------------------------------
template <typename GS, typename GRP, typename OUT>
__device__ inline int equipartition_bounds_t(const GS* gs, const GRP* grp, int G, int n, int Y,
                                             OUT* bounds) {
  // n <= 2^29, so every quantity below fits 32-bit integers
  int R0 = 0, g0 = 0, row = 1;
  bounds[0] = 0;
  while (true) {
    const int mult = Y - row + 1;
    const int thr = 2 * (n - R0);
    const int Tp = 2 * R0 + (thr + mult - 1) / mult;
    int ps = (Tp - 1) >> 1;
    if (ps > n - 1) ps = n - 1;
    int gc = (int)grp[ps];
    if (gc < g0 + 1) gc = g0 + 1;
    if (gc >= G) break;
    if ((int)gs[gc] + (int)gs[gc + 1] < Tp) {
      ++gc;
      if (gc >= G) break;
    }
    R0 = (int)gs[gc];
    g0 = gc;
    bounds[row] = (OUT)R0;
    ++row;
  }
  bounds[row] = (OUT)n;
  return row;
}

__device__ inline int equipartition_bounds(const int* gs, const int* grp, int G, int n, int Y,
                                           int* bounds) {
  return equipartition_bounds_t<int, int, int>(gs, grp, G, n, Y, bounds);
}



// khat = max(floor(c * floor(B / y)), 1) (Appendix item 7: khat = c x)
__host__ __device__ __forceinline__ int khat_of(int B, int y, double c) {
  const int x = B / y;
  const int k = (int)floor(c * (double)x);
  return k < 1 ? 1 : k;
}

// Record of one task written by the partition kernel (int32 units, a
// multiple of 4): header (k, yhat, clumps, 0, H(Q) as double), superclump
// ends c_0..c_k, counts cum[r][t] for r < yhat.  Sized for the largest k and
// yhat a task with row count y can have in a batch of n samples, B = B(n).
__host__ __device__ __forceinline__ int64_t rec_size(int B, int n, double c, int y) {
  int kk = khat_of(B, y, c);
  if (kk > n) kk = n;
  const int64_t sz = 6 + (int64_t)(kk + 1) * (y + 1);
  return (sz + 3) & ~int64_t(3);
}

__host__ __device__ __forceinline__ int64_t rec_offset(int B, int n, double c, int y) {
  int64_t off = 0;
  for (int yy = 2; yy < y; ++yy) off += rec_size(B, n, c, yy);
  return off;
}

// Copies the first nint ints of a task record to shared memory with 16-byte
// loads, four in flight per thread (threads tid, tid + T, ... of a group of
// T).  Records start on 16-byte boundaries and are padded to a multiple of
// 4 ints, so the rounded-up copy stays inside the record.
__device__ __forceinline__ void copy_record(int* __restrict__ dst, const int32_t* __restrict__ src,
                                            int nint, int tid, int T) {
  const int n4 = (nint + 3) >> 2;
  const int4* __restrict__ s4 = reinterpret_cast<const int4*>(src);
  int4* __restrict__ d4 = reinterpret_cast<int4*>(dst);
  for (int i0 = tid; i0 < n4; i0 += 4 * T) {
    int4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q * T < n4) v[q] = s4[i0 + q * T];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q * T < n4) d4[i0 + q * T] = v[q];
  }
}

// first cell of row count y in the y-major layout of M
__device__ __forceinline__ int row_offset(int B, int y) {
  int off = 0;
  for (int yy = 2; yy < y; ++yy) off += B / yy - 1;
  return off;
}

// ---------------------------------------------------------------------------
// Kernel parameter blocks
// ---------------------------------------------------------------------------

// Per-slot rank data.  A slot is a clean variable (slot = variable index) or
// one side of a pair with missing samples (slot >= p, compacted samples).
struct RankData {
  int32_t* perm;     // [slots][n] sorted position -> sample
  int32_t* pos;      // [slots][n] sample -> sorted position
  int32_t* grp;      // [slots][n] sorted position -> tie group
  int32_t* gstart;   // [slots][n+1] group starts
  int32_t* ngroups;  // [slots]
  int32_t* nslot;    // [slots] samples in the slot
  int64_t stride;    // n
};

struct EquiData {
  int32_t* bounds;   // [slots][R][bstride] row starts, sorted positions
  int32_t* yhat;     // [slots][R]
  int R;             // row counts y = 2 .. R + 1
  int bstride;       // R + 2
};

struct PairPrep {
  int32_t* slot;     // [chunk][2] slot of X and of Y
  int32_t* n_used;   // [chunk]
  int32_t* B;        // [chunk]
  int32_t* flags;    // [chunk] status bits (1 << GMINE_E_*)
  int32_t* dirty;    // [chunk] chunk-local indices of pairs with their own ranks
  int32_t* ndirty;   // [1]
  const int32_t* order;   // [pairs] batch position -> pair index (NULL: identity)
  const uint8_t* aidx;    // [pairs] B table of each pair (NULL: table 0)
  int64_t btab_stride;    // ints per B table (n + 1)
  int64_t slot0;          // first slot of the pairs with their own ranks
  int all_dirty;          // every pair gets its own compacted ranks
};

// Index of the pair at batch position i (pairs may be processed in a
// planned order), and its B(m) table.
__device__ __forceinline__ int64_t pair_index(const PairPrep& pp, int64_t i) {
  return pp.order ? (int64_t)pp.order[i] : i;
}
__device__ __forceinline__ const int32_t* btab_of(const int32_t* Btab, const PairPrep& pp,
                                                  int64_t pair) {
  return Btab + (pp.aidx ? (int64_t)pp.aidx[pair] * pp.btab_stride : 0);
}

struct PartParams {
  RankData rk;
  EquiData eq;
  PairPrep pp;
  const double* L64;   // [n+1] m ln m
  const double* lnt;   // [n+1] ln m
  int32_t* rec;        // task records, [chunk][2][rec_per_orient] ints
  int64_t rec_per_orient;
  int B_full, n_full;  // B and n of the full sample count
  double c;
  int64_t chunk_pairs;
  const int64_t* rec_off;     // [B/2+2] first int of row count y's record
  unsigned long long* queue;  // atomic job counter: (part, pair, orientation)
  int parts;                  // CTAs per (pair, orientation), row counts interleaved
  int off_pi, off_gU;  // shared by the CTA: [n] uint16 each
  int off_warps;       // first per-warp region
  int warp_smem;       // bytes of shared memory per warp
  int off_Qs, off_q, off_cgrp, off_cstart, off_scb, off_mixed, off_eb;  // within a warp region
  unsigned char* gscr;   // when set, the regions above live here (per CTA), not in shared memory
  int64_t gscr_per_cta;
};

// Rows of the global R table a warp of the blocked DP stages in shared
// memory at a time, and the bytes of its buffer (R rows of up to 160 bytes,
// then superclump rows of up to 32 bytes).
constexpr int kDPStageRows = 16;
constexpr int kDPStageBytes = kDPStageRows * (160 + 32);

struct DPParams {
  PairPrep pp;
  const int32_t* rec;
  int64_t rec_per_orient;
  const int64_t* rec_off;  // [B/2+2] first int of row count y's record
  int B_full, n_full;
  double c;
  const double* L64;
  const float* L32;
  const double* lnt;
  double* Mo;          // [chunk][2][cells_max] normalised M_o per orientation
  int cells_max;
  int64_t chunk_pairs;
  int64_t task_begin, task_end;  // tasks of this launch
  unsigned long long* queue;
  int64_t* counters;             // [2] DP candidates, tasks (may be NULL)
  char* scratch;                 // per-CTA R tables that do not fit in smem
  int64_t scratch_per_cta;
  gmine_trace trace;
  int64_t trace_pair0, trace_npairs;
};

// Shared-memory layout of the warp-per-task DP kernel (byte offsets): the
// CTA's entropy table, then one region per warp.
struct SmallPlan {
  int off_L, off_warps, warp_smem;
  int off_E, off_W, off_A, off_rec, off_I, off_cuts;  // within a warp region
  int LW;     // row stride of the W / A tables (levels 0..xmax)
  int total;
};

// Shared-memory layout of the warp-per-task blocked DP kernel (byte
// offsets): the CTA's entropy table, then one region per warp.
struct WarpPlan {
  int off_L, off_warps, warp_smem;
  int off_R, off_sd, off_rbuf, off_Rtop, off_lst, off_I, off_cuts;  // within a warp region
  int LS;     // row stride of the R table (the level group: every level a
              // lane's running maxima read lies inside the row)
  int xmax;   // largest x of the launch
  int total;
};

// Shared-memory layout of the level-major DP kernel (byte offsets).
struct MidPlan {
  int off_E, off_R, off_L, off_rec, off_I, off_cuts, off_ecol;
  int KS;     // row stride of the level-major R table (t = 0..kmax)
  int xmax;
  int total;
};

// Shared-memory layout of the DP kernel (byte offsets).
struct DPPlan {
  int off_R, off_Rtop, off_X, off_Eb, off_rbuf, off_L, off_sd;
  int off_Eb2;  // a second in-block triangle (double buffering), or -1
  int off_stage;  // per-warp staging buffers of R rows (R table in global memory)
  int64_t sd_scr_off;  // off_sd < 0: the superclump rows live in the CTA's global scratch here
  int64_t x_scr_off;   // off_X < 0: the X buffers live in the CTA's global scratch here
  int off_tb;          // traceback scratch (cuts, I(l), l*(l)): the X region, or its own
  int64_t cuts_scr_off;  // >= 0: the traceback's path buffers in the CTA's global scratch here
  int64_t scr_bytes;   // global scratch per CTA (0 when the R table is in shared memory)
  int off_I_rel, off_lst_rel;  // within the traceback scratch
  int LS;     // row stride of the R table: source levels 1..lmax-1, mult. of 4
  int LX;     // row stride of the X buffers: levels 1..lmax, odd (the lanes'
              // rows then start in distinct shared-memory banks)
  int xmax;   // largest x of the launch
  int total;
};

struct FinalParams {
  const double* Mo;
  int cells_max;
  PairPrep pp;
  int64_t chunk_pairs;
  int64_t pair0;
  gmine_pair_score* scores;
  double* M;           // may be NULL
  int64_t m_stride;
  const int32_t* eq_yhat;  // [slots][R] rows used per (slot, y)
  int R;
};

}  // namespace gm
