// k_dp_small.cu -- the OptimizeXAxis dynamic program for tasks with few
// columns (x <= 9, small superclump counts), one warp per task.
//
// The recursion is the method's own (SOM Algorithm 2; Appendix item 10):
//   W(t,1) = -E(0,t),  W(t,l) = max_{s in [l-1, t]} W(s,l-1) - E(s,t)
// with s = t an empty last column (E(t,t) = 0), the first maximum in
// increasing s chosen, computed t after t.  For each t the warp first forms
// the entropy column E(., t) (Appendix item 10b), then every level: lanes
// are split into (level, phase) groups, phase p scanning s = l-1+p, l-1+p+P,
// ..., and a few shuffles combine the phases (larger value, else smaller s).
// The argument table A(t,l) is kept, so the chosen partitions follow
// directly.  The plain path keeps the table in double; the float path
// re-scores each chosen partition in double.
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

template <typename real>
__device__ __forceinline__ real ninf_of();
template <>
__device__ __forceinline__ float ninf_of<float>() { return __int_as_float(0xff800000); }
template <>
__device__ __forceinline__ double ninf_of<double>() {
  return __longlong_as_double((long long)0xfff0000000000000ull);
}

template <typename real>
__device__ __forceinline__ real E_small(const real* __restrict__ Lt, const int* __restrict__ scb,
                                        const int* __restrict__ cum, int ks, int yhat, int s, int t) {
  real e = Lt[scb[t] - scb[s]];
  const int* __restrict__ ct = cum + t;
  const int* __restrict__ cs = cum + s;
  int r = 0;
  // four rows at a time: the loads run ahead, the subtractions keep the
  // order of increasing r
  for (; r + 4 <= yhat; r += 4) {
    const real l0 = Lt[ct[(r + 0) * ks] - cs[(r + 0) * ks]];
    const real l1 = Lt[ct[(r + 1) * ks] - cs[(r + 1) * ks]];
    const real l2 = Lt[ct[(r + 2) * ks] - cs[(r + 2) * ks]];
    const real l3 = Lt[ct[(r + 3) * ks] - cs[(r + 3) * ks]];
    e -= l0;
    e -= l1;
    e -= l2;
    e -= l3;
  }
  for (; r < yhat; ++r) e -= Lt[ct[r * ks] - cs[r * ks]];
  return e;
}

template <typename real>
__global__ void __launch_bounds__(128) k_dp_small(DPParams P, SmallPlan S) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr bool fp32 = sizeof(real) == 4;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int LW = S.LW;
  unsigned char* my = sm + S.off_warps + (int64_t)wib * S.warp_smem;
  real* W = reinterpret_cast<real*>(my + S.off_W);             // [kmax+1][LW]
  int16_t* A = reinterpret_cast<int16_t*>(my + S.off_A);       // [kmax+1][LW]
  real* Ecol = reinterpret_cast<real*>(my + S.off_Ecol);       // [kmax+1]
  int* scb = reinterpret_cast<int*>(my + S.off_scb);           // [kmax+1]
  int* cum = reinterpret_cast<int*>(my + S.off_cum);           // [cum_max]
  real* Vb = reinterpret_cast<real*>(my + S.off_V);            // [LW]
  int* Va = reinterpret_cast<int*>(my + S.off_Va);             // [LW]
  double* Iw = reinterpret_cast<double*>(my + S.off_I);        // [LW]
  int* cuts = reinterpret_cast<int*>(my + S.off_cuts);         // [LW][LW]
  const real* Lt;
  {
    const real* Lsrc;
    if constexpr (fp32) Lsrc = P.L32; else Lsrc = P.L64;
    real* Ls = reinterpret_cast<real*>(sm + S.off_L);
    for (int m = threadIdx.x; m <= P.n_full; m += blockDim.x) Ls[m] = Lsrc[m];
    Lt = Ls;
  }
  __syncthreads();
  const real NINF = ninf_of<real>();
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
                         rec_offset(P.B_full, P.n_full, P.c, y);
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
    const int x = B / y;
    const int ks = k + 1;
    const int lmax = min(x, k);
    for (int j = lane; j <= k; j += 32) scb[j] = rec[6 + j];
    for (int i = lane; i < yhat * ks; i += 32) cum[i] = rec[6 + ks + i];
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = lane; j <= k; j += 32) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncwarp();

    if (k >= 2) {
      // lanes as (level, phase): LP level groups of P phases
      const int nlev = lmax - 1;
      const int LP = nlev <= 1 ? 1 : nlev <= 2 ? 2 : nlev <= 4 ? 4 : 8;
      const int Pph = 32 / LP;
      const int li = lane / Pph;
      const int ph = lane - li * Pph;
      const int lv = 2 + li;  // this lane's level
      // entropy columns double-buffered: column t+1 is formed before the
      // levels of t are reduced, so its loads overlap that work
      real* const Ec0 = Ecol;
      real* const Ec1 = Ecol + S.LE;
      if (lane == 0) Ec1[0] = E_small<real>(Lt, scb, cum, ks, yhat, 0, 1);
      __syncwarp();
      for (int t = 1; t <= k; ++t) {
        const real* Et = (t & 1) ? Ec1 : Ec0;
        if (t < k) {
          real* En = (t & 1) ? Ec0 : Ec1;
          for (int s = lane; s <= t; s += 32) En[s] = E_small<real>(Lt, scb, cum, ks, yhat, s, t + 1);
        }
        const int lt = min(t, lmax);
        real best = NINF;
        int arg = 0x7fffffff;
        if (lv <= lt) {
          for (int s = lv - 1 + ph; s < t; s += Pph) {
            const real v = W[s * LW + (lv - 1)] - Et[s];
            if (v > best) {
              best = v;
              arg = s;
            }
          }
        }
        for (int d = Pph >> 1; d > 0; d >>= 1) {
          const real ob = __shfl_xor_sync(0xffffffffu, best, d);
          const int oa = __shfl_xor_sync(0xffffffffu, arg, d);
          if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
          }
        }
        if (ph == 0 && lv <= lt) {
          Vb[lv] = best;
          Va[lv] = arg;
        }
        __syncwarp();
        if (lane == 0) {
          real cur = -Et[0];  // W(t,1)
          W[t * LW + 1] = cur;
          A[t * LW + 1] = 0;
          for (int l = 2; l <= lt; ++l) {
            const real v = Vb[l];
            int a;
            if (cur > v) {  // s = t: W(t,l-1) - E(t,t) is the larger
              a = t;
            } else {
              cur = v;
              a = Va[l];
            }
            W[t * LW + l] = cur;
            A[t * LW + l] = (int16_t)a;
          }
        }
        __syncwarp();
      }
      // chosen partitions: lane l-2 follows A back from (k, l)
      const int l = 2 + lane;
      if (l <= lmax) {
        int* cut = cuts + (l - 2) * LW;
        int tcur = k;
        for (int v = l; v >= 2; --v) {
          const int s = A[tcur * LW + v];
          cut[v - 2] = s;
          tcur = s;
        }
        double I;
        if constexpr (fp32) {
          // re-score in double, in the DP's own order
          int prev = 0;
          double w = 0.0;
          for (int c = 0; c < l; ++c) {
            const int bnd = c == l - 1 ? k : cut[c];
            double e = P.L64[scb[bnd] - scb[prev]];
            for (int r = 0; r < yhat; ++r) e -= P.L64[cum[r * ks + bnd] - cum[r * ks + prev]];
            w = c == 0 ? -e : w - e;
            prev = bnd;
          }
          I = HQ + w / (double)n;
        } else {
          I = HQ + (double)W[k * LW + l] / (double)n;
        }
        Iw[l] = I;
        if (P.trace.d_cuts) {
          int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
          for (int c = 0; c < l - 1; ++c) dst[c] = cut[c];
        }
      }
      __syncwarp();
    }
    const int rowoff = row_offset(B, y);
    double* Mo = P.Mo + ((int64_t)pl * 2 + o) * P.cells_max + rowoff;
    for (int l = 2 + lane; l <= x; l += 32) {
      const double I = k <= 1 ? 0.0 : Iw[min(l, k)];
      const int mn = min(l, yhat);
      Mo[l - 2] = mn < 2 ? 0.0 : I / P.lnt[mn];
      if (P.trace.d_I) P.trace.d_I[trace_task * P.trace.I_stride + (l - 2)] = I;
      if (P.trace.d_cuts && (l > k || k <= 1)) {
        int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
        for (int c = 0; c < l - 1; ++c) dst[c] = -1;
      }
    }
    if (lane == 0 && yhat < 2) atomicOr(&P.pp.flags[pl], 1 << GMINE_E_CONSTANT);
    if (lane == 0 && k >= 2 && lmax >= 2) {
      const long long L = lmax, K = k;
      long long cand = (L + 1) * L * (L - 1) / 6;
      const long long tsum = (K * (K + 1) - L * (L + 1)) / 2;
      cand += (L - 1) * tsum - (K - L) * (L - 1) * L / 2;
      cand_sum += cand;
    }
    if (lane == 0) ++task_sum;
    __syncwarp();
  }
  if (lane == 0 && P.counters && task_sum > 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(P.counters), (unsigned long long)cand_sum);
    atomicAdd(reinterpret_cast<unsigned long long*>(P.counters) + 1, (unsigned long long)task_sum);
  }
}

template <typename real>
static cudaError_t small_cfg(int smem, int threads, int* blocks) {
  const cudaError_t e =
      cudaFuncSetAttribute(k_dp_small<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_dp_small<real>, threads, smem);
}

cudaError_t dp_small_configure(bool fp32, int smem, int threads, int* blocks_per_sm) {
  return fp32 ? small_cfg<float>(smem, threads, blocks_per_sm)
              : small_cfg<double>(smem, threads, blocks_per_sm);
}

cudaError_t dp_small_occupancy(bool fp32, int smem, int threads, int* blocks_per_sm) {
  return fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_small<float>, threads, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_small<double>, threads, smem);
}

cudaError_t dp_small_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                            const DPParams& P, const SmallPlan& S) {
  if (fp32)
    k_dp_small<float><<<grid, threads, smem, st>>>(P, S);
  else
    k_dp_small<double><<<grid, threads, smem, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace gm
