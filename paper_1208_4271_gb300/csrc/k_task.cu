// k_task.cu -- one CTA per task (pair, orientation o, row count y), popped
// from an atomic queue by a persistent grid.  Per task:
//   Q of the row variable (EquipartitionYAxis, precomputed per slot) in the
//   column variable's order; GetClumpsPartition; GetSuperclumpsPartition
//   with khat = c * floor(B/y); per-superclump prefix counts cum[r][t] and
//   H(Q) (Appendix item 10a); the OptimizeXAxis DP over the superclumps
//   with the entropy column E(., t) of each t (Appendix item 10b); the
//   normalised row of M_o (Appendix item 4).
// The DP runs in double (plain path) or in float with exact int32 counts,
// each chosen partition then re-scored in double.
#include <cfloat>

#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

__device__ __forceinline__ void argmax_combine(double& b, int& a, double ob, int oa) {
  if (ob > b || (ob == b && oa < a)) {
    b = ob;
    a = oa;
  }
}
__device__ __forceinline__ void argmax_combine(float& b, int& a, float ob, int oa) {
  if (ob > b || (ob == b && oa < a)) {
    b = ob;
    a = oa;
  }
}

template <typename real>
__device__ __forceinline__ real neg_inf();
template <>
__device__ __forceinline__ double neg_inf<double>() { return __longlong_as_double(0xfff0000000000000ll); }
template <>
__device__ __forceinline__ float neg_inf<float>() { return __int_as_float(0xff800000); }

// E(s,t) in double, summed as L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s])
// with increasing r (Appendix item 10b).
__device__ __forceinline__ double entropy_term64(const double* __restrict__ L64,
                                                 const int* scb, const int* cum,
                                                 int ks, int yhat, int s, int t) {
  double e = L64[scb[t] - scb[s]];
  for (int r = 0; r < yhat; ++r) e -= L64[cum[r * ks + t] - cum[r * ks + s]];
  return e;
}

template <typename real>
__global__ void __launch_bounds__(256)
k_task(TaskParams P, SmemPlan S) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_task;
  __shared__ int s_k;
  __shared__ double s_HQ;
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int NW = T >> 5;
  const bool fp32 = sizeof(real) == 4;
  char* scratch = P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta;
  const int R = P.eq.R;
  const int64_t C = P.chunk_pairs;
  const int64_t st = P.rk.stride;

  // scratch layout per CTA: [region P][DP tables][int argmax][cuts]
  unsigned char* pbase = S.p_in_smem ? sm : reinterpret_cast<unsigned char*>(scratch);
  char* wscratch = scratch + S.scratch_P;
  uint16_t* Qs = reinterpret_cast<uint16_t*>(pbase + S.offP_Qs);
  uint16_t* q = reinterpret_cast<uint16_t*>(pbase + S.offP_q);
  uint8_t* mixed = reinterpret_cast<uint8_t*>(pbase + S.offP_mixed);
  uint8_t* cflag = reinterpret_cast<uint8_t*>(pbase + S.offP_cflag);
  int* grpU = reinterpret_cast<int*>(pbase + S.offP_grpU);
  int* cgrp = reinterpret_cast<int*>(pbase + S.offP_cgrp);
  int* cstart = reinterpret_cast<int*>(pbase + S.offP_cstart);
  int* eb = reinterpret_cast<int*>(sm + S.offK_eb);
  int* scb = reinterpret_cast<int*>(sm + S.offK_scb);
  int* cum = reinterpret_cast<int*>(sm + S.offK_cum);
  real* Ecol = reinterpret_cast<real*>(sm + S.offK_Ecol);
  real* Vb = reinterpret_cast<real*>(sm + S.offK_V);
  int* Va = reinterpret_cast<int*>(sm + S.offK_Varg);
  int* tmp = reinterpret_cast<int*>(sm + S.offK_tmp);

  const real* Lr;
  if constexpr (sizeof(real) == 4) Lr = P.L32; else Lr = P.L64;

  for (;;) {
    if (tid == 0) s_task = (long long)atomicAdd(P.queue, 1ull);
    __syncthreads();
    const int64_t task = s_task;
    __syncthreads();
    if (task >= P.ntasks) break;

    const int r = 2 + (int)(task / (2 * C));
    const int o = (int)((task / C) % 2);
    const int64_t pl = task % C;
    const int n = P.pp.n_used[pl];
    const int B = P.pp.B[pl];
    const int64_t trace_task =
        ((int64_t)(r - 2) * 2 + o) * P.trace_npairs + P.trace_pair0 + pl;

    if (n < 4 || B < 4 || r > B / 2) {
      if (tid == 0) {
        if (P.trace.d_k) P.trace.d_k[trace_task] = 0;
        if (P.trace.d_yhat) P.trace.d_yhat[trace_task] = 0;
        if (P.trace.d_clumps) P.trace.d_clumps[trace_task] = 0;
      }
      continue;
    }
    const int sU = P.pp.slot[2 * pl + o];
    const int sV = P.pp.slot[2 * pl + (1 - o)];
    const int x = B / r;
    const int khat = khat_of(B, r, P.c);
    const int yhat = P.eq.yhat[(int64_t)sV * R + (r - 2)];
    const int32_t* gb = P.eq.bounds + ((int64_t)sV * R + (r - 2)) * P.eq.bstride;

    // 1-2. rows of the V-sorted positions
    for (int j = tid; j <= yhat; j += T) eb[j] = gb[j];
    __syncthreads();
    for (int p = tid; p < n; p += T) {
      int lo = 0, hi = yhat;  // largest j with eb[j] <= p
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (eb[mid] <= p) lo = mid; else hi = mid;
      }
      Qs[p] = (uint16_t)lo;
    }
    // 3. Q in U order, U's tie groups
    const int32_t* permU = P.rk.perm + (int64_t)sU * st;
    const int32_t* posV = P.rk.pos + (int64_t)sV * st;
    const int32_t* grpUg = P.rk.grp + (int64_t)sU * st;
    const int GU = P.rk.ngroups[sU];
    for (int g = tid; g < GU; g += T) mixed[g] = 0;
    __syncthreads();
    for (int m = tid; m < n; m += T) {
      q[m] = Qs[posV[permU[m]]];
      grpU[m] = grpUg[m];
    }
    __syncthreads();
    // 4. x-tie runs with mixed rows (Algorithm GetClumpsPartition, first pass)
    for (int m = 1 + tid; m < n; m += T)
      if (grpU[m] == grpU[m - 1] && q[m] != q[m - 1]) mixed[grpU[m]] = 1;
    __syncthreads();
    // 5. a clump starts where the (relabelled) row label changes
    for (int m = tid; m < n; m += T) {
      int f;
      if (m == 0) f = 1;
      else if (grpU[m] == grpU[m - 1]) f = 0;
      else f = (mixed[grpU[m]] | mixed[grpU[m - 1]] | (q[m] != q[m - 1])) ? 1 : 0;
      cflag[m] = (uint8_t)f;
      cgrp[m] = f;
    }
    __syncthreads();
    const int nc = block_exclusive_scan(cgrp, n, tmp);
    for (int m = tid; m < n; m += T) {
      const int e = cgrp[m];
      const int f = cflag[m];
      cgrp[m] = e + f - 1;
      if (f) cstart[e] = m;
    }
    if (tid == 0) cstart[nc] = n;
    __syncthreads();
    // 6. superclumps (Algorithm GetSuperclumpsPartition)
    const bool superclump = nc > khat;
    if (superclump) {
      if (tid == 0) s_k = equipartition_bounds(cstart, cgrp, nc, n, khat, scb);
    } else {
      for (int j = tid; j <= nc; j += T) scb[j] = cstart[j];
      if (tid == 0) s_k = nc;
    }
    __syncthreads();
    const int k = s_k;
    const int ks = k + 1;
    // 7. cell counts per (row, superclump), then prefix over superclumps
    for (int i = tid; i < yhat * ks; i += T) cum[i] = 0;
    __syncthreads();
    for (int m = tid; m < n; m += T) {
      int t;
      if (superclump) {
        int lo = 0, hi = k;  // largest t with scb[t] <= m
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (scb[mid] <= m) lo = mid; else hi = mid;
        }
        t = lo;
      } else {
        t = cgrp[m];
      }
      atomicAdd(&cum[(int)q[m] * ks + t + 1], 1);
    }
    __syncthreads();
    for (int rr = warp; rr < yhat; rr += NW) {
      int carry = 0;
      for (int base = 0; base < ks; base += 32) {
        const int i = base + lane;
        const int v = i < ks ? cum[rr * ks + i] : 0;
        int incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int oo = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += oo;
        }
        if (i < ks) cum[rr * ks + i] = carry + incl;
        carry += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    // 8. H(Q) = ln n - sum_r L(q_r) / n
    if (tid == 0) {
      double sL = 0.0;
      for (int rr = 0; rr < yhat; ++rr) sL += P.L64[cum[rr * ks + k]];
      s_HQ = P.lnt[n] - sL / (double)n;
    }

    // 9. OptimizeXAxis DP: W(t,1) = -E(0,t);
    //    W(t,l) = max_{s in [l-1, t]} W(s,l-1) - E(s,t), first maximum wins.
    const int lmax = min(x, k);
    real* W;
    int* A32 = nullptr;      // argmax table, double path with trace
    int16_t* A16 = nullptr;  // argmax table, float path
    const int64_t welems = (int64_t)(lmax + 1) * ks;
    if (P.w_in_smem) {
      W = reinterpret_cast<real*>(sm);
      if (fp32) A16 = reinterpret_cast<int16_t*>(sm + ((welems * sizeof(real) + 15) & ~15ll));
    } else {
      W = reinterpret_cast<real*>(wscratch);
      if (fp32) A16 = reinterpret_cast<int16_t*>(wscratch + ((welems * sizeof(real) + 15) & ~15ll));
    }
    char* scr2 = wscratch + S.scratch_tables;  // past the global DP tables
    if (!fp32 && P.trace.d_cuts) A32 = reinterpret_cast<int*>(scr2);
    int* cutbuf = reinterpret_cast<int*>(scr2 + S.scratch_A32);
    __syncthreads();

    for (int t = 1; t <= k; ++t) {
      for (int s = tid; s < t; s += T) {
        real e = Lr[scb[t] - scb[s]];
        for (int rr = 0; rr < yhat; ++rr) e -= Lr[cum[rr * ks + t] - cum[rr * ks + s]];
        Ecol[s] = e;
      }
      __syncthreads();
      const int lt = min(t, lmax);
      for (int l = 2 + warp; l <= lt; l += NW) {
        real best = neg_inf<real>();
        int arg = 0x7fffffff;
        const real* Wl = W + (int64_t)(l - 1) * ks;
        for (int s = l - 1 + lane; s <= t - 1; s += 32) {
          const real v = Wl[s] - Ecol[s];
          if (v > best) {
            best = v;
            arg = s;
          }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const real ob = __shfl_xor_sync(0xffffffffu, best, d);
          const int oa = __shfl_xor_sync(0xffffffffu, arg, d);
          argmax_combine(best, arg, ob, oa);
        }
        if (lane == 0) {
          Vb[l] = best;
          Va[l] = arg;
        }
      }
      __syncthreads();
      if (tid == 0) {
        W[ks + t] = -Ecol[0];
        if (A32) A32[ks + t] = 0;
        if (A16) A16[ks + t] = 0;
        for (int l = 2; l <= lt; ++l) {
          const real cand_t = W[(int64_t)(l - 1) * ks + t];  // s = t: empty column
          real w;
          int a;
          if (cand_t > Vb[l]) {
            w = cand_t;
            a = t;
          } else {
            w = Vb[l];
            a = Va[l];
          }
          W[(int64_t)l * ks + t] = w;
          if (A32) A32[(int64_t)l * ks + t] = a;
          if (A16) A16[(int64_t)l * ks + t] = (int16_t)a;
        }
      }
      __syncthreads();
    }

    // 10. I(l), trace, normalised M_o(l, r)
    const double HQ = s_HQ;
    const int rowoff = row_offset(B, r);
    double* Mo = P.Mo + ((int64_t)pl * 2 + o) * P.cells_max + rowoff;
    const bool want_cuts = fp32 || (P.trace.d_cuts != nullptr);
    for (int l = 2 + tid; l <= x; l += T) {
      double I;
      int* cut = cutbuf + (l - 2) * (l - 1) / 2;
      if (k <= 1) {
        I = 0.0;
      } else {
        const int lc = min(l, k);
        if (want_cuts) {
          int tt = k;
          for (int ll = lc; ll >= 2; --ll) {
            const int s = fp32 ? (int)A16[(int64_t)ll * ks + tt] : A32[(int64_t)ll * ks + tt];
            cut[ll - 2] = s;
            tt = s;
          }
        }
        if (fp32) {
          // re-score the chosen partition in double, in the DP's own order
          int prev = 0;
          double w = 0.0;
          for (int j = 0; j < lc - 1; ++j) {
            const int s = cut[j];
            const double e = entropy_term64(P.L64, scb, cum, ks, yhat, prev, s);
            w = (j == 0) ? -e : w - e;
            prev = s;
          }
          const double e = entropy_term64(P.L64, scb, cum, ks, yhat, prev, k);
          w = (lc - 1 == 0) ? -e : w - e;
          I = HQ + w / (double)n;
        } else {
          I = HQ + (double)W[(int64_t)lc * ks + k] / (double)n;
        }
      }
      const int mn = min(l, yhat);
      Mo[l - 2] = mn < 2 ? 0.0 : I / P.lnt[mn];
      if (P.trace.d_I) P.trace.d_I[trace_task * P.trace.I_stride + (l - 2)] = I;
      if (P.trace.d_cuts) {
        int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
        for (int j = 0; j < l - 1; ++j) dst[j] = (l <= k && k > 1) ? cut[j] : -1;
      }
    }
    if (tid == 0) {
      if (yhat < 2) atomicOr(&P.pp.flags[pl], 1 << GMINE_E_CONSTANT);
      if (P.trace.d_k) P.trace.d_k[trace_task] = k;
      if (P.trace.d_yhat) P.trace.d_yhat[trace_task] = yhat;
      if (P.trace.d_clumps) P.trace.d_clumps[trace_task] = nc;
    }
    if (P.trace.d_sc_ends && k + 1 <= P.trace.sc_stride)
      for (int j = tid; j <= k; j += T) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = scb[j];
    __syncthreads();
  }
}

// Host-side wrappers: the kernel templates are instantiated and launched in
// this translation unit only.
cudaError_t task_configure(bool fp32, int smem, int threads, int* blocks_per_sm) {
  cudaError_t e;
  if (fp32) {
    e = cudaFuncSetAttribute(k_task<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_task<float>, threads, smem);
  }
  e = cudaFuncSetAttribute(k_task<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_task<double>, threads, smem);
}

cudaError_t task_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                        const TaskParams& P, const SmemPlan& S) {
  if (fp32)
    k_task<float><<<grid, threads, smem, st>>>(P, S);
  else
    k_task<double><<<grid, threads, smem, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace gm
