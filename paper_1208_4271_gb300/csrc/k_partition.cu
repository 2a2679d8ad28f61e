// k_partition.cu -- the partitions of every task (pair, orientation o, row
// count y): the row variable's EquipartitionYAxis map in the column
// variable's order, GetClumpsPartition, GetSuperclumpsPartition with
// khat = c * floor(B/y), the per-superclump prefix counts cum[r][t] and H(Q)
// (Appendix items 5-7 and 10a, the two algorithm listings).
//
// One CTA per (pair, o): the map pi[m] = position in the row variable's
// order of the m-th point in the column variable's order, and the column
// variable's tie groups, are gathered once into shared memory and serve all
// row counts; each warp then takes row counts y one after another.  The
// result of every task is a record in global memory that the DP kernels
// read:
//   int32 [0] k, [1] yhat, [2] clumps, [3] unused, [4..5] H(Q) as double,
//   [6 .. 6+k] superclump ends c_0..c_k (sorted positions),
//   then cum[r][t] for r < yhat, t = 0..k (row-major, stride k+1).
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

// samples per lane whose loads a per-sample loop issues together
constexpr int kBatch = 4;

__device__ __forceinline__ bool bit_of(const uint32_t* bm, int g) {
  return (bm[g >> 5] >> (g & 31)) & 1u;
}

// EquipartitionYAxis over the clumps (cstart[g] = P_g, the first position
// of clump g; cstart[nc] = n): with the current row (superclump) number
// `row` starting at position R0, the next one starts at the first clump g
// after the current row's first clump with
//   (P_g + P_{g+1} - 2 R0) (khat - row + 1) >= 2 (n - R0),
// the exact integer form of 2# + |S| >= 2d; the left side grows with g.  If
// there is none, the rest of the clumps form the last row.  Writes the row
// starts scb[0..rows-1] and scb[rows] = n and returns rows.
template <bool WIDE>
__device__ __forceinline__ bool row_ends_at(int Sg, int R0, int mult, int rhs) {
  if constexpr (WIDE) return (long long)(Sg - 2 * R0) * mult >= rhs;
  else return (Sg - 2 * R0) * mult >= rhs;
}

// One thread, clump after clump, the clump starts loaded eight at a time
// ahead of the tests: for few clumps per row, where the warp's per-row
// ballot, find-first and shuffle would cost more than a compare per clump.
template <bool WIDE, typename IT>
__device__ int superclump_rows_seq(const IT* __restrict__ cstart, int nc, int n, int khat,
                                   IT* __restrict__ scb) {
  constexpr int kAhead = 8;
  int R0 = 0, row = 1;
  scb[0] = 0;
  int mult = khat, rhs = 2 * n;
  int Pg = cstart[1];
  for (int g = 1; g < nc; g += kAhead) {
    int Pn[kAhead];
#pragma unroll
    for (int j = 0; j < kAhead; ++j) Pn[j] = g + 1 + j <= nc ? (int)cstart[g + 1 + j] : n;
#pragma unroll
    for (int j = 0; j < kAhead; ++j) {
      const int Pj = j == 0 ? Pg : Pn[j - 1];
      if (g + j < nc && row_ends_at<WIDE>(Pj + Pn[j], R0, mult, rhs)) {
        R0 = Pj;
        scb[row] = (IT)R0;
        ++row;
        mult = khat - row + 1;
        rhs = 2 * (n - R0);
      }
    }
    Pg = Pn[kAhead - 1];
  }
  scb[row] = (IT)n;
  return row;
}

// The warp tests 32 clumps at a time; two warp-wide minimum reductions give
// every lane the first hit and its start.
template <bool WIDE, typename IT>
__device__ int superclump_rows_warp(const IT* __restrict__ cstart, int nc, int n, int khat,
                                    IT* __restrict__ scb, int lane) {
  int R0 = 0, g0 = 0, row = 1;
  if (lane == 0) scb[0] = 0;
  for (;;) {
    const int mult = khat - row + 1;
    const int rhs = 2 * (n - R0);
    int found = -1, Pf = 0;
    for (int gb = g0 + 1; gb < nc; gb += 32) {
      const int g = gb + lane;
      int Pg = 0;
      bool ok = false;
      if (g < nc) {
        Pg = cstart[g];
        ok = row_ends_at<WIDE>(Pg + (int)cstart[g + 1], R0, mult, rhs);
      }
      // the first clump that ends the row, and its start (the starts grow
      // with g, so the smallest start among the hits is the first one's)
      const unsigned fg = __reduce_min_sync(0xffffffffu, ok ? (unsigned)g : 0xffffffffu);
      const unsigned fp = __reduce_min_sync(0xffffffffu, ok ? (unsigned)Pg : 0xffffffffu);
      if (fg != 0xffffffffu) {
        found = (int)fg;
        Pf = (int)fp;
        break;
      }
    }
    if (found < 0) break;  // the rest of the clumps form the last row
    R0 = Pf;
    g0 = found;
    if (lane == 0) scb[row] = (IT)R0;
    ++row;
  }
  if (lane == 0) scb[row] = (IT)n;
  return row;
}

template <bool GLOBAL, typename IT>
__global__ void __launch_bounds__(128) k_partition_t(PartParams P) {
  extern __shared__ __align__(16) unsigned char smd[];
  // the CTA's regions: shared memory, or (large n) this CTA's global scratch
  // (a template parameter, so that the shared instance keeps shared-memory
  // addressing)
  unsigned char* sm = GLOBAL ? P.gscr + (int64_t)blockIdx.x * P.gscr_per_cta : smd;
  __shared__ long long s_job;
  __shared__ int s_y;                    // next row count of the current (pair, o)
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  IT* pi = reinterpret_cast<IT*>(sm + P.off_pi);   // [n] U position -> V position
  IT* gU = reinterpret_cast<IT*>(sm + P.off_gU);   // [n] U position -> tie group
  unsigned char* my = sm + P.off_warps + (int64_t)wib * P.warp_smem;
  IT* Qs = reinterpret_cast<IT*>(my + P.off_Qs);     // V position -> row
  IT* cnt = reinterpret_cast<IT*>(my + P.off_Qs);    // counts (aliases Qs)
  IT* q = reinterpret_cast<IT*>(my + P.off_q);       // U position -> row
  IT* cgrp = reinterpret_cast<IT*>(my + P.off_cgrp); // U position -> clump
  IT* cstart = reinterpret_cast<IT*>(my + P.off_cstart);
  IT* scb = reinterpret_cast<IT*>(my + P.off_scb);
  uint32_t* mixed = reinterpret_cast<uint32_t*>(my + P.off_mixed);
  int* eb = reinterpret_cast<int*>(my + P.off_eb);

  const int64_t C = P.chunk_pairs;
  const int R = P.eq.R;
  const int64_t st = P.rk.stride;
  for (;;) {
    if (threadIdx.x == 0) {
      s_job = (long long)atomicAdd(P.queue, 1ull);
      s_y = 0;
    }
    __syncthreads();
    const int64_t job = s_job;
    __syncthreads();
    // job = part * 2C + (pair * 2 + o): with P.parts > 1 several CTAs share a
    // (pair, o), part j taking the row counts y = 2 + j, 2 + j + parts, ...
    // (the first parts, with the heavy small y, come first)
    if (job >= 2 * C * P.parts) break;
    const int part = (int)(job / (2 * C));
    const int64_t pj = job - (int64_t)part * 2 * C;
    const int64_t pl = pj >> 1;
    const int o = (int)(pj & 1);
    const int n = P.pp.n_used[pl];
    const int B = P.pp.B[pl];
    int32_t* rec0 = P.rec + ((int64_t)pl * 2 + o) * P.rec_per_orient;
    if (n < 4 || B < 4) {
      for (int y = 2 + part + P.parts * (int)threadIdx.x; y <= P.B_full / 2; y += P.parts * blockDim.x) {
        int32_t* rec = rec0 + P.rec_off[y];
        rec[0] = 0;
        rec[1] = 0;
        rec[2] = 0;
      }
      continue;
    }
    const int sU = P.pp.slot[2 * pl + o];
    const int sV = P.pp.slot[2 * pl + (1 - o)];
    const int32_t* permU = P.rk.perm + (int64_t)sU * st;
    const int32_t* posV = P.rk.pos + (int64_t)sV * st;
    const int32_t* grpU = P.rk.grp + (int64_t)sU * st;
    const int GU = P.rk.ngroups[sU];
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
      pi[m] = (IT)posV[permU[m]];
      gU[m] = (IT)grpU[m];
    }
    __syncthreads();

    // row counts taken in increasing order (the long superclump chains of
    // the small y first) by whichever warp is free
    for (;;) {
      int yy = 0;
      if (lane == 0) yy = 2 + part + P.parts * atomicAdd(&s_y, 1);
      const int y = __shfl_sync(0xffffffffu, yy, 0);
      if (y > P.B_full / 2) break;
      int32_t* rec = rec0 + P.rec_off[y];
      if (y > B / 2) {  // fewer samples than the batch's n: no such task
        if (lane == 0) {
          rec[0] = 0;
          rec[1] = 0;
          rec[2] = 0;
        }
        continue;
      }
      const int yhat = P.eq.yhat[(int64_t)sV * R + (y - 2)];
      const int32_t* gb = P.eq.bounds + ((int64_t)sV * R + (y - 2)) * P.eq.bstride;
      for (int j = lane; j <= yhat; j += 32) eb[j] = gb[j];
      const bool ties = GU < n;  // else every tie run is one point: none is mixed
      if (ties)
        for (int w = lane; w < (GU + 31) / 32; w += 32) mixed[w] = 0u;
      __syncwarp();
      // rows of the V-sorted positions (row r holds [eb[r], eb[r+1]);
      // eb[yhat] = n), then of the U-sorted positions
      for (int r = 0; r < yhat; ++r) {
        const int b1 = eb[r + 1];
#pragma unroll 4
        for (int p = eb[r] + lane; p < b1; p += 32) Qs[p] = (IT)r;
      }
      __syncwarp();
      // (the loops over samples take kBatch of a lane's samples at a time,
      // loads first: the stores into the same shared memory would otherwise
      // keep the next sample's loads from starting early)
      for (int m0 = lane; m0 < n; m0 += 32 * kBatch) {
        int pv[kBatch];
        IT qv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) pv[u] = m0 + 32 * u < n ? (int)pi[m0 + 32 * u] : 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) qv[u] = Qs[pv[u]];
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (m0 + 32 * u < n) q[m0 + 32 * u] = qv[u];
      }
      __syncwarp();
      // x-tie runs whose rows are mixed get one fresh label (Algorithm
      // GetClumpsPartition, first pass; one label per run)
      if (ties)
        for (int m = 1 + lane; m < n; m += 32) {
          const int g = gU[m];
          if (g == gU[m - 1] && q[m] != q[m - 1]) atomicOr(&mixed[g >> 5], 1u << (g & 31));
        }
      __syncwarp();
      // a clump starts where the label changes (second pass): ballot per 32
      int nc = 0;
      for (int base = 0; base < n; base += 32 * kBatch) {
        bool f[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int m = base + 32 * u + lane;
          f[u] = false;
          if (m < n) {
            if (m == 0) {
              f[u] = true;
            } else {
              if (ties) {
                const int g = gU[m], gp = gU[m - 1];
                f[u] = g != gp && (bit_of(mixed, g) || bit_of(mixed, gp) || q[m] != q[m - 1]);
              } else {
                f[u] = q[m] != q[m - 1];
              }
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int m = base + 32 * u + lane;
          const unsigned mask = __ballot_sync(0xffffffffu, f[u]);
          const int before = __popc(mask & ((1u << lane) - 1u));
          if (m < n) {
            cgrp[m] = (IT)(nc + before + (f[u] ? 1 : 0) - 1);
            if (f[u]) cstart[nc + before] = (IT)m;
          }
          nc += __popc(mask);
        }
      }
      if (lane == 0) cstart[nc] = (IT)n;
      __syncwarp();
      // superclumps: EquipartitionYAxis over the clumps (Algorithm
      // GetSuperclumpsPartition), one row after another
      const int khat = khat_of(B, y, P.c);
      int k;
      const bool superclump = nc > khat;
      if (superclump) {
        // (the products reach (2n) * khat: 64-bit where that passes 2^31)
        const bool wide = 2LL * n * khat >= (1LL << 31);
        int rows;
        if (nc <= 3 * khat) {  // (y = 2..3 at n = 1340, B = 75, c = 15)
          int r1 = 0;
          if (lane == 0) r1 = wide ? superclump_rows_seq<true>(cstart, nc, n, khat, scb)
                                   : superclump_rows_seq<false>(cstart, nc, n, khat, scb);
          rows = __shfl_sync(0xffffffffu, r1, 0);
        } else {
          rows = wide ? superclump_rows_warp<true>(cstart, nc, n, khat, scb, lane)
                      : superclump_rows_warp<false>(cstart, nc, n, khat, scb, lane);
        }
        k = rows;
      } else {
        for (int j = lane; j <= nc; j += 32) scb[j] = cstart[j];
        k = nc;
      }
      const int ks = k + 1;
      __syncwarp();
      // superclump of every clump (cstart is free once the superclumps are
      // known): a clump lies inside one superclump
      IT* sc_of = cstart;
      if (superclump) {
        for (int t = lane; t < k; t += 32) {
          const int c0 = cgrp[scb[t]], c1 = cgrp[scb[t + 1] - 1];
          for (int c = c0; c <= c1; ++c) sc_of[c] = (IT)t;
        }
      }
      // counts: 16 bits each, two per 32-bit word (n < 65536), or 32 bits
      constexpr int per_word = 4 / (int)sizeof(IT);
      for (int i = lane; i < (yhat * ks + per_word - 1) / per_word; i += 32)
        reinterpret_cast<uint32_t*>(cnt)[i] = 0u;
      __syncwarp();
      for (int m0 = lane; m0 < n; m0 += 32 * kBatch) {
        int ci[kBatch], ti[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const bool in = m0 + 32 * u < n;
          ci[u] = in ? (int)cgrp[m0 + 32 * u] : 0;
          ti[u] = in ? (int)q[m0 + 32 * u] : -1;  // row, -1 past the end
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) ci[u] = superclump ? (int)sc_of[ci[u]] : ci[u];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (ti[u] < 0) continue;
          const int i = ti[u] * ks + ci[u] + 1;
          if constexpr (sizeof(IT) == 2)
            atomicAdd(reinterpret_cast<uint32_t*>(cnt) + (i >> 1), 1u << (16 * (i & 1)));
          else
            atomicAdd(reinterpret_cast<uint32_t*>(cnt) + i, 1u);
        }
      }
      __syncwarp();
      // prefix over superclumps, written to the record; row totals give H(Q)
      int32_t* rcum = rec + 6 + ks;
      double sL = 0.0;
      if (yhat >= 8) {
        // many rows: lanes over rows, each row's prefix in place (counts
        // <= n fit the index type), row totals into eb (free after the fill), the
        // record written coalesced; the L(total) loads side by side, summed
        // in increasing r
        for (int r = lane; r < yhat; r += 32) {
          IT* row = cnt + r * ks;
          int run = 0;
          int t = 0;
          for (; t + kBatch <= ks; t += kBatch) {  // the loads ahead of the stores
            int a[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) a[u] = row[t + u];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
              run += a[u];
              row[t + u] = (IT)run;
            }
          }
          for (; t < ks; ++t) {
            run += row[t];
            row[t] = (IT)run;
          }
          eb[r] = run;
        }
        __syncwarp();
        for (int i = lane; i < yhat * ks; i += 32) rcum[i] = cnt[i];
        for (int r0 = 0; r0 < yhat; r0 += 32) {
          const double Lr = r0 + lane < yhat ? P.L64[eb[r0 + lane]] : 0.0;
          const int nr = min(32, yhat - r0);
          for (int j = 0; j < nr; ++j) sL += __shfl_sync(0xffffffffu, Lr, j);
        }
      } else
      for (int r = 0; r < yhat; ++r) {
        int carry = 0;
        // kBatch chunks of 32 scanned side by side, then stored with the
        // carry in order
        for (int base = 0; base < ks; base += 32 * kBatch) {
          int incl[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int i = base + 32 * u + lane;
            incl[u] = i < ks ? (int)cnt[r * ks + i] : 0;
          }
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
              const int oo = __shfl_up_sync(0xffffffffu, incl[u], d);
              if (lane >= d) incl[u] += oo;
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            const int i = base + 32 * u + lane;
            if (i < ks) rcum[r * ks + i] = carry + incl[u];
            carry += __shfl_sync(0xffffffffu, incl[u], 31);
          }
        }
        sL += P.L64[carry];  // increasing r, as H(Q) is defined
      }
      for (int j = lane; j <= k; j += 32) rec[6 + j] = scb[j];
      if (lane == 0) {
        rec[0] = k;
        rec[1] = yhat;
        rec[2] = nc;
        rec[3] = 0;
        *reinterpret_cast<double*>(rec + 4) = P.lnt[n] - sL / (double)n;
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

cudaError_t partition_configure(bool global, bool wide, int smem, int threads, int* blocks_per_sm) {
  auto k = wide ? k_partition_t<true, uint32_t>
                : (global ? k_partition_t<true, uint16_t> : k_partition_t<false, uint16_t>);
  cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t partition_launch(bool global, bool wide, int grid, int threads, int smem,
                             cudaStream_t st, const PartParams& P) {
  if (wide)
    k_partition_t<true, uint32_t><<<grid, threads, smem, st>>>(P);
  else if (global)
    k_partition_t<true, uint16_t><<<grid, threads, smem, st>>>(P);
  else
    k_partition_t<false, uint16_t><<<grid, threads, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace gm
