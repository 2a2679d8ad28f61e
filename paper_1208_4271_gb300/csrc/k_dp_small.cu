// k_dp_small.cu -- the OptimizeXAxis dynamic program for tasks with few
// columns (3 <= x <= 9) and few superclumps, one warp per task, level after
// level.
//
// The recursion is the method's own (SOM Algorithm 2; Appendix item 10):
//   W(t,1) = -E(0,t),  W(t,l) = max_{s in [l-1, t]} W(s,l-1) - E(s,t)
// with s = t an empty last column (E(t,t) = 0) and the first maximum in
// increasing s chosen.  The warp first forms the whole entropy triangle
// E(s,t), s < t (Appendix item 10b), every lane busy, then takes the levels
// one after another: within a level every t is independent, lanes over t,
// each lane scanning s upwards and keeping the argument A(t,l).  W(t,l) is
// needed for t >= l (a source of level l+1 has s >= l) and, at the last
// level, only at t = k: that cell is one warp-wide argmax.  The chosen
// partitions follow from A.  The plain path keeps W in double; the float
// path re-scores each chosen partition in double.
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

// a > b and a == b for the values the W recursion compares (W, W - E with
// E >= +0, -inf), which lie in [-inf, -0.0]: doubles through their bit
// patterns on the integer pipe (on that range the order of the patterns is
// the reverse of the order of the values), floats directly.
__device__ __forceinline__ bool gt_neg(float a, float b) { return a > b; }
__device__ __forceinline__ bool gt_neg(double a, double b) {
  return (unsigned long long)__double_as_longlong(a) < (unsigned long long)__double_as_longlong(b);
}
__device__ __forceinline__ bool eq_neg(float a, float b) { return a == b; }
__device__ __forceinline__ bool eq_neg(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}

namespace {

template <typename real>
__device__ __forceinline__ real ninf_of();
template <>
__device__ __forceinline__ float ninf_of<float>() { return __int_as_float(0xff800000); }
template <>
__device__ __forceinline__ double ninf_of<double>() {
  return __longlong_as_double((long long)0xfff0000000000000ull);
}

// E(s,t) = L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s]), increasing r
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

// E(s_q, t_q) for NE entries with their loads interleaved: NE independent
// chains per lane, each in increasing r
template <typename real, int NE>
__device__ __forceinline__ void E_smallN(const real* __restrict__ Lt, const int* __restrict__ scb,
                                         const int* __restrict__ cum, int ks, int yhat,
                                         const int (&s)[NE], const int (&t)[NE], real (&e)[NE]) {
#pragma unroll
  for (int q = 0; q < NE; ++q) e[q] = Lt[scb[t[q]] - scb[s[q]]];
  int r = 0;
  for (; r + 4 <= yhat; r += 4) {
    real l[NE][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < NE; ++q) l[q][u] = Lt[cum[(r + u) * ks + t[q]] - cum[(r + u) * ks + s[q]]];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < NE; ++q) e[q] -= l[q][u];
  }
  for (; r < yhat; ++r) {
    real l[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) l[q] = Lt[cum[r * ks + t[q]] - cum[r * ks + s[q]]];
#pragma unroll
    for (int q = 0; q < NE; ++q) e[q] -= l[q];
  }
}

// offset of E(s, .) in the packed triangle: row s holds t = s+1 .. k
__device__ __forceinline__ int tri_row(int s, int k) { return s * k - (s * (s - 1)) / 2; }

}  // namespace

template <typename real>
__global__ void __launch_bounds__(128) k_dp_small(DPParams P, SmallPlan S) {
  extern __shared__ __align__(16) unsigned char sm[];
  constexpr bool fp32 = sizeof(real) == 4;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int LW = S.LW;
  unsigned char* my = sm + S.off_warps + (int64_t)wib * S.warp_smem;
  real* Et = reinterpret_cast<real*>(my + S.off_E);            // packed triangle
  real* W = reinterpret_cast<real*>(my + S.off_W);             // [kmax+1][LW]
  int16_t* A = reinterpret_cast<int16_t*>(my + S.off_A);       // [kmax+1][LW]
  int* recb = reinterpret_cast<int*>(my + S.off_rec);          // the task's record
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
    const int x = B / y;
    const int ks = k + 1;
    const int lmax = min(x, k);
    copy_record(recb, rec, 6 + ks + yhat * ks, lane, 32);
    const int* scb = recb + 6;      // superclump ends
    const int* cum = recb + 6 + ks;  // cum[r][t] at r * ks + t
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = lane; j <= k; j += 32) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncwarp();

    if (k >= 2) {
      // ---- the entropy triangle: entry f = tri_row(s,k) + t - s - 1 in
      // lane f mod 32, four entries (f, f + 32, ...) at a time, (s, t)
      // advancing along the rows
      {
        const int npairs = k * (k + 1) / 2;
        int s = 0, pos = lane;  // pos = t - s - 1 within row s (k - s entries)
        auto advance = [&](int d) {
          pos += d;
          while (s < k && pos >= k - s) {
            pos -= k - s;
            ++s;
          }
        };
        advance(0);
        constexpr int NE = 4;  // entries in flight per lane
        for (int f = lane; f < npairs; f += 32 * NE) {
          int sq[NE], tq[NE];
#pragma unroll
          for (int q = 0; q < NE; ++q) {
            const bool live = f + 32 * q < npairs;
            sq[q] = live ? s : sq[0];
            tq[q] = live ? s + 1 + pos : tq[0];
            advance(32);
          }
          real e[NE];
          E_smallN<real, NE>(Lt, scb, cum, ks, yhat, sq, tq, e);
#pragma unroll
          for (int q = 0; q < NE; ++q)
            if (f + 32 * q < npairs) Et[f + 32 * q] = e[q];
        }
      }
      __syncwarp();
      // ---- W(t,1) = -E(0,t)
      for (int t = 1 + lane; t <= k; t += 32) {
        W[t * LW + 1] = -Et[t - 1];
        A[t * LW + 1] = 0;
      }
      __syncwarp();
      // ---- levels 2 .. lmax-1 at every t >= l: lanes over t, s upwards
      for (int l = 2; l < lmax; ++l) {
        for (int t0 = l; t0 <= k; t0 += 32) {
          const int t = t0 + lane;
          const int tt = min(t, k);
          real best = NINF;
          int arg = l - 1;
          const int s_hi = min(t0 + 31, k);  // the warp's bound: s < the largest t
          if constexpr (fp32) {
            // E(s, tt) at tri_row(s, k) + tt - s - 1, which grows by k - s - 1
            // from s to s + 1; W(s, l-1) a row further (measured: -4 % on the
            // float launches, +1 % on the double ones, which keep the plain form)
            int eo = tri_row(l - 1, k) + tt - l;
            const real* wp = W + (l - 1) * LW + (l - 1);
#pragma unroll 4
            for (int s = l - 1; s < s_hi; ++s) {
              const real v = *wp - Et[eo];
              if (s < t && gt_neg(v, best)) {
                best = v;
                arg = s;
              }
              eo += k - s - 1;
              wp += LW;
            }
          } else {
            for (int s = l - 1; s < s_hi; ++s) {
              const real v = W[s * LW + (l - 1)] - Et[tri_row(s, k) + tt - s - 1];
              if (s < t && gt_neg(v, best)) {
                best = v;
                arg = s;
              }
            }
          }
          if (t <= k) {
            const real wt = W[t * LW + (l - 1)];  // s = t, the empty column
            if (gt_neg(wt, best)) {
              best = wt;
              arg = t;
            }
            W[t * LW + l] = best;
            A[t * LW + l] = (int16_t)arg;
          }
        }
        __syncwarp();
      }
      // ---- the last level at t = k only: lanes over s, the first maximum
      {
        const int l = lmax;
        real best = NINF;
        int arg = 0x7fffffff;
        for (int s = l - 1 + lane; s <= k; s += 32) {
          const real wv = W[s * LW + (l - 1)];
          const real v = s < k ? wv - Et[tri_row(s, k) + k - s - 1] : wv;
          if (gt_neg(v, best)) {
            best = v;
            arg = s;
          }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const real ob = __shfl_xor_sync(0xffffffffu, best, d);
          const int oa = __shfl_xor_sync(0xffffffffu, arg, d);
          if (gt_neg(ob, best) || (eq_neg(ob, best) && oa < arg)) {
            best = ob;
            arg = oa;
          }
        }
        if (lane == 0) {
          W[k * LW + l] = best;
          A[k * LW + l] = (int16_t)arg;
        }
      }
      __syncwarp();
      // ---- chosen partitions: lane l-2 follows A back from (k, l)
      {
        const int l = 2 + lane;
        if (l <= lmax) {
          int* cut = cuts + (l - 2) * LW;
          int tcur = k;
          for (int v = l; v >= 2; --v) {
            const int s = A[tcur * LW + v];
            cut[v - 2] = s;
            tcur = s;
          }
          if constexpr (!fp32) Iw[l] = HQ + (double)W[k * LW + l] / (double)n;
          if (P.trace.d_cuts) {
            int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
            for (int c = 0; c < l - 1; ++c) dst[c] = cut[c];
          }
        }
      }
      __syncwarp();
      if constexpr (fp32) {
        // re-score each chosen partition in double: the terms (column c,
        // row r) over the lanes, then a warp sum
        for (int l = 2; l <= lmax; ++l) {
          const int* cut = cuts + (l - 2) * LW;
          const int nt = l * (yhat + 1);
          double part = 0.0;
          for (int i = lane; i < nt; i += 32) {
            const int c = i / (yhat + 1), r = i - c * (yhat + 1);
            const int a = c == 0 ? 0 : cut[c - 1];
            const int b = c == l - 1 ? k : cut[c];
            // -E(a,b) = -L(c_b - c_a) + sum_r L(cum[r][b] - cum[r][a])
            part += r == 0 ? -P.L64[scb[b] - scb[a]]
                           : P.L64[cum[(r - 1) * ks + b] - cum[(r - 1) * ks + a]];
          }
#pragma unroll
          for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
          if (lane == 0) Iw[l] = HQ + part / (double)n;
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
      // the W candidates formed: the levels below the last at every t >= l,
      // the last at t = k
      long long cand = 0;
      for (int l = 2; l < lmax; ++l) cand += (long long)(k - l + 1) * (k - l + 2) / 2;
      cand += k - lmax + 2;
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
      allow_dynamic_smem(reinterpret_cast<const void*>(k_dp_small<real>), smem);
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
