// k_dp_two.cu -- the OptimizeXAxis dynamic program for tasks with two
// columns (x = floor(B/y) = 2), one warp per task.
//
// With x = 2 the method's recursion (SOM Algorithm 2; Appendix item 10)
// only needs its last cell:
//   W(s,1) = -E(0,s),   W(k,2) = max_{s in [1, k]} W(s,1) - E(s,k),
// s = k being an empty second column (E(k,k) = 0), the first maximum in
// increasing s chosen.  So a task needs the 2k entropies E(0,s) and E(s,k)
// instead of the whole entropy matrix: the warp stages the task record in
// shared memory and lane s forms both from column s (rows 0 and k are
// broadcasts), in increasing r as E is defined.  I(2) = H(Q) + W(k,2)/n.
// The plain path does this in double; the float path picks s in float and
// re-scores the chosen partition in double.
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

namespace {

template <typename real>
struct TwoBits;
template <>
struct TwoBits<float> {
  __device__ static float ninf() { return __int_as_float(0xff800000); }
};
template <>
struct TwoBits<double> {
  __device__ static double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
};

// E(a, b) from the record (ends at rec+6, cum row r at rec+6+ks+r*ks), the
// table L in shared memory; rows in increasing r, four loads in flight.
template <typename real>
__device__ __forceinline__ real entropy_rec(const real* __restrict__ L, const int32_t* __restrict__ ends,
                                            const int32_t* __restrict__ cum, int ks, int yhat, int a,
                                            int b) {
  real e = L[ends[b] - ends[a]];
  int r = 0;
  for (; r + 4 <= yhat; r += 4) {
    const int d0 = cum[(r + 0) * ks + b] - cum[(r + 0) * ks + a];
    const int d1 = cum[(r + 1) * ks + b] - cum[(r + 1) * ks + a];
    const int d2 = cum[(r + 2) * ks + b] - cum[(r + 2) * ks + a];
    const int d3 = cum[(r + 3) * ks + b] - cum[(r + 3) * ks + a];
    const real l0 = L[d0], l1 = L[d1], l2 = L[d2], l3 = L[d3];
    e -= l0;
    e -= l1;
    e -= l2;
    e -= l3;
  }
  for (; r < yhat; ++r) e -= L[cum[r * ks + b] - cum[r * ks + a]];
  return e;
}

}  // namespace

template <typename real>
__global__ void __launch_bounds__(256, 2) k_dp_two(DPParams P, int off_rec, int rec_bytes) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr bool fp32 = sizeof(real) == 4;
  const int lane = threadIdx.x & 31;
  real* Lt = reinterpret_cast<real*>(sm);  // [n+1]
  int* recb = reinterpret_cast<int*>(sm + off_rec + (threadIdx.x >> 5) * rec_bytes);  // the warp's record
  {
    const real* Lsrc;
    if constexpr (fp32) Lsrc = P.L32; else Lsrc = P.L64;
    for (int m = threadIdx.x; m <= P.n_full; m += blockDim.x) Lt[m] = Lsrc[m];
  }
  __syncthreads();
  const int64_t C = P.chunk_pairs;
  long long cand_sum = 0, task_sum = 0;

  for (;;) {
    long long tk = 0;
    if (lane == 0) tk = (long long)atomicAdd(P.queue, 1ull);
    const int64_t task = __shfl_sync(0xffffffffu, tk, 0) + P.task_begin;
    if (task >= P.task_end) break;
    const int y = 2 + (int)(task / (2 * C));
    const int o = (int)((task / C) % 2);
    const int64_t pl = task % C;
    const int n = P.pp.n_used[pl];
    const int B = P.pp.B[pl];
    const int32_t* rec = P.rec + ((int64_t)pl * 2 + o) * P.rec_per_orient +
                         P.rec_off[y];
    const int64_t trace_task = ((int64_t)(y - 2) * 2 + o) * P.trace_npairs + P.trace_pair0 + pl;
    const bool valid = n >= 4 && B >= 4 && y <= B / 2;
    const int k = valid ? rec[0] : 0;
    const int yhat = valid ? rec[1] : 0;
    if (lane == 0 && P.trace.d_k) {
      P.trace.d_k[trace_task] = k;
      if (P.trace.d_yhat) P.trace.d_yhat[trace_task] = yhat;
      if (P.trace.d_clumps) P.trace.d_clumps[trace_task] = valid ? rec[2] : 0;
    }
    if (!valid) continue;
    const double HQ = *reinterpret_cast<const double*>(rec + 4);
    const int x = B / y;  // 2 for every task of this kernel's launches
    const int ks = k + 1;
    copy_record(recb, rec, 6 + ks + yhat * ks, lane, 32);
    const int32_t* ends = recb + 6;
    const int32_t* cum = recb + 6 + ks;
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = lane; j <= k; j += 32) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncwarp();

    double I = 0.0;
    int scut = k;
    if (k >= 2 && x >= 2) {
      // candidates W(s,1) - E(s,k) for s < k, and W(k,1) for s = k
      real best = TwoBits<real>::ninf();
      int arg = 0x7fffffff;
      for (int s0 = 1; s0 <= k; s0 += 32) {
        const int s = s0 + lane;
        if (s <= k) {
          const real w1 = -entropy_rec<real>(Lt, ends, cum, ks, yhat, 0, s);
          const real cand = s < k ? w1 - entropy_rec<real>(Lt, ends, cum, ks, yhat, s, k) : w1;
          if (cand > best) {  // increasing s per lane: the first maximum
            best = cand;
            arg = s;
          }
        }
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const real ob = __shfl_xor_sync(0xffffffffu, best, d);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, d);
        if (ob > best || (ob == best && oa < arg)) {
          best = ob;
          arg = oa;
        }
      }
      scut = arg;
      if constexpr (fp32) {
        // re-score the chosen partition in double, -E(0,s) - E(s,k): the
        // terms (column, row) over the lanes, then a warp sum
        const int ncol = scut < k ? 2 : 1;
        double part = 0.0;
        for (int i = lane; i < ncol * (yhat + 1); i += 32) {
          const int c = i / (yhat + 1), r = i - c * (yhat + 1);
          const int a = c == 0 ? 0 : scut;
          const int b = c == ncol - 1 ? k : scut;
          part += r == 0 ? -P.L64[ends[b] - ends[a]]
                         : P.L64[cum[(r - 1) * ks + b] - cum[(r - 1) * ks + a]];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        I = HQ + part / (double)n;
      } else {
        I = HQ + (double)best / (double)n;
      }
      cand_sum += k;
    }
    if (lane == 0) {
      double* Mo = P.Mo + ((int64_t)pl * 2 + o) * P.cells_max + row_offset(B, y);
      for (int l = 2; l <= x; ++l) {
        const double Il = k <= 1 ? 0.0 : I;
        const int mn = min(l, yhat);
        Mo[l - 2] = mn < 2 ? 0.0 : Il / P.lnt[mn];
        if (P.trace.d_I) P.trace.d_I[trace_task * P.trace.I_stride + (l - 2)] = Il;
        if (P.trace.d_cuts) {
          int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
          for (int c = 0; c < l - 1; ++c) dst[c] = k <= 1 ? -1 : scut;
        }
      }
      if (yhat < 2) atomicOr(&P.pp.flags[pl], 1 << GMINE_E_CONSTANT);
      ++task_sum;
    }
    __syncwarp();
  }
  if (lane == 0 && P.counters && task_sum > 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(P.counters), (unsigned long long)cand_sum);
    atomicAdd(reinterpret_cast<unsigned long long*>(P.counters) + 1, (unsigned long long)task_sum);
  }
}

cudaError_t dp_two_configure(bool fp32, int smem, int threads, int* blocks_per_sm) {
  cudaError_t e;
  if (fp32) {
    e = allow_dynamic_smem(reinterpret_cast<const void*>(k_dp_two<float>), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_two<float>, threads, smem);
  }
  e = allow_dynamic_smem(reinterpret_cast<const void*>(k_dp_two<double>), smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_two<double>, threads, smem);
}

cudaError_t dp_two_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                          const DPParams& P, int off_rec, int rec_bytes) {
  if (fp32)
    k_dp_two<float><<<grid, threads, smem, st>>>(P, off_rec, rec_bytes);
  else
    k_dp_two<double><<<grid, threads, smem, st>>>(P, off_rec, rec_bytes);
  return cudaGetLastError();
}

}  // namespace gm
