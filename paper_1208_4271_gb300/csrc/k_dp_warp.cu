// k_dp_warp.cu -- the OptimizeXAxis dynamic program (SOM Algorithm 2 with
// the precomputations of Appendix item 10) for tasks with a moderate number
// of levels, one warp per task, float path.
//
// The recursion is the one of k_dp.cuh without empty columns,
//   R(t,1) = -E(0,t),  R(t,l) = max_{s in [l-1, t-1]} R(s,l-1) - E(s,t),
// whose prefix maximum over levels is the method's W(t,l).  t runs in blocks
// of 32, lane j owning t = t0 + j, and one warp takes a block in two steps:
//   A: every s below the block: E(s,t) once per (s, t), then the running
//      maxima of all LEV levels in registers (the R row of s is a warp-wide
//      16-byte broadcast), two subtractions per packed instruction and two
//      s per three-operand max;
//   B: s inside the block, level after level: lane j keeps E(t0+i, t0+j),
//      i < j, in registers and reads the 32 values R(t0+i, l-1) of the level
//      below as eight 16-byte broadcasts.
// With one warp per task nothing waits on a barrier and the partial maxima
// never leave the registers; the latency of step B and of the traceback is
// covered by the other warps' tasks.  The last level is needed at t = k
// only.  The chosen partitions are recovered by the traceback of k_dp.cuh
// (an exact match of R(s, lv-1) - E(s, t) with R(t, lv), scanning down from
// t - 1) and re-scored in double.  R, E and the candidates are the same
// floats as in k_dp.cuh and k_dp_mid.cu, so the three kernels choose the
// same partitions (the re-scored sums may differ in the last bits, their
// terms being added in another order).
#include "k_dp.cuh"

namespace gm {

namespace {

// E(s,t) for a fixed t whose row td (yhat <= TDW - 1) sits in registers:
// row s comes in 16-byte broadcast loads, terms in increasing r.
template <int TDW>
__device__ __forceinline__ float entropy_w(const float* __restrict__ Lt, const int* __restrict__ sd,
                                           int SW, int yhat, const int (&td)[TDW], int s) {
  if constexpr (TDW == 8) {
    return entropy_reg<float>(Lt, sd, SW, yhat, td, s);
  } else {
    const int4* row = reinterpret_cast<const int4*>(sd + s * SW);
    const int4 a = row[0];
    float e = Lt[td[0] - a.x];
    if (yhat > 0) e -= Lt[td[1] - a.y];
    if (yhat > 1) e -= Lt[td[2] - a.z];
    if (yhat > 2) e -= Lt[td[3] - a.w];
#pragma unroll
    for (int q = 1; q < TDW / 4; ++q) {
      if (yhat > 4 * q - 1) {
        const int4 b = row[q];
        e -= Lt[td[4 * q + 0] - b.x];
        if (yhat > 4 * q + 0) e -= Lt[td[4 * q + 1] - b.y];
        if (yhat > 4 * q + 1) e -= Lt[td[4 * q + 2] - b.z];
        if (yhat > 4 * q + 2) e -= Lt[td[4 * q + 3] - b.w];
      }
    }
    return e;
  }
}

}  // namespace

template <int LEV, int TDW>
__global__ void __launch_bounds__(224, 2) k_dp_warp(DPParams P, WarpPlan S) {
  using BT = Bits<float>;
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* my = sm + S.off_warps + (int64_t)wib * S.warp_smem;
  float* Rt = reinterpret_cast<float*>(my + S.off_R);      // [kmax+1][LS]: R(t,l) at column l-1
  int* sd = reinterpret_cast<int*>(my + S.off_sd);         // s-major superclump rows
  float* rbuf = reinterpret_cast<float*>(my + S.off_rbuf);  // [2][32]
  float* Rtop = reinterpret_cast<float*>(my + S.off_Rtop);  // R(k, lmax)
  int* lst = reinterpret_cast<int*>(my + S.off_lst);        // [xmax+1]
  double* Iw = reinterpret_cast<double*>(my + S.off_I);     // [xmax+1]
  int* cuts = reinterpret_cast<int*>(my + S.off_cuts);      // [8][xmax]
  const int LS = S.LS;
  const float* Lt;
  {
    float* Ls = reinterpret_cast<float*>(sm + S.off_L);
    for (int m = threadIdx.x; m <= P.n_full; m += blockDim.x) Ls[m] = P.L32[m];
    Lt = Ls;
  }
  __syncthreads();
  const float NINF = BT::ninf();
  const float PINF = __int_as_float(0x7f800000);
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
    const int32_t* rec = P.rec + ((int64_t)pl * 2 + o) * P.rec_per_orient + P.rec_off[y];
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
    const int SW = sd_width(yhat);
    // record (ends, then cum row-major) -> s-major rows, a row per lane;
    // unused columns 0
    for (int j = lane; j <= k; j += 32) {
      int* row = sd + j * SW;
      for (int c4 = 0; c4 < SW; c4 += 4) {
        int4 v;
        v.x = c4 + 0 <= yhat ? rec[6 + (c4 + 0) * ks + j] : 0;
        v.y = c4 + 1 <= yhat ? rec[6 + (c4 + 1) * ks + j] : 0;
        v.z = c4 + 2 <= yhat ? rec[6 + (c4 + 2) * ks + j] : 0;
        v.w = c4 + 3 <= yhat ? rec[6 + (c4 + 3) * ks + j] : 0;
        *reinterpret_cast<int4*>(row + c4) = v;
      }
    }
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = lane; j <= k; j += 32) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncwarp();
    auto Rget = [&](int t, int l) -> float { return l == lmax ? *Rtop : Rt[t * LS + (l - 1)]; };

    if (k >= 2) {
      {
        float4* R4 = reinterpret_cast<float4*>(Rt);
        const float4 n4 = make_float4(NINF, NINF, NINF, NINF);
        for (int i = lane; i < ks * LS / 4; i += 32) R4[i] = n4;
      }
      if (lane == 0) *Rtop = NINF;
      __syncwarp();
      for (int t = 1 + lane; t <= k; t += 32) Rt[t * LS] = -entropy_term<float>(Lt, sd, SW, yhat, 0, t);
      __syncwarp();

      const int nb = (k + 31) / 32;
      for (int b = 0; b < nb; ++b) {
        const int t0 = 1 + 32 * b;
        const int t = t0 + lane;
        const bool tv = t <= k;
        const int tt = tv ? t : k;
        int td[TDW];
#pragma unroll
        for (int c = 0; c < TDW; ++c) td[c] = c < SW ? sd[tt * SW + c] : 0;
        float acc[LEV];
#pragma unroll
        for (int i = 0; i < LEV; ++i) acc[i] = NINF;
        // ---- A: s in [1, t0 - 1] (an even count), levels 2 .. LEV+1
        if (t0 > 1) {
          float e0 = entropy_w<TDW>(Lt, sd, SW, yhat, td, 1);
          float e1 = entropy_w<TDW>(Lt, sd, SW, yhat, td, 2);
#pragma unroll 1
          for (int s = 1; s < t0; s += 2) {
            const bool more = s + 2 < t0;
            const float n0 = more ? entropy_w<TDW>(Lt, sd, SW, yhat, td, s + 2) : e0;
            const float n1 = more ? entropy_w<TDW>(Lt, sd, SW, yhat, td, s + 3) : e1;
            const float* R0 = Rt + s * LS;
            const float* R1 = R0 + LS;
            const unsigned long long ee0 = splat_x2(e0), ee1 = splat_x2(e1);
#pragma unroll
            for (int g = 0; g < LEV / 4; ++g) {
              const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(R0 + 4 * g);
              const ulonglong2 c = *reinterpret_cast<const ulonglong2*>(R1 + 4 * g);
              const float2 a0 = sub_x2(a.x, ee0), a1 = sub_x2(a.y, ee0);
              const float2 c0 = sub_x2(c.x, ee1), c1 = sub_x2(c.y, ee1);
              acc[4 * g + 0] = fmax3(acc[4 * g + 0], a0.x, c0.x);
              acc[4 * g + 1] = fmax3(acc[4 * g + 1], a0.y, c0.y);
              acc[4 * g + 2] = fmax3(acc[4 * g + 2], a1.x, c1.x);
              acc[4 * g + 3] = fmax3(acc[4 * g + 3], a1.y, c1.y);
            }
            e0 = n0;
            e1 = n1;
          }
        }
        // ---- B: s inside the block
        // the in-block column E(t0+i, t0+lane), i < lane, in registers.
        // Lane j < 16 pairs with lane 31 - j (31 entries between them): in
        // step q < 16 the high lane forms its own entry i = q, the low lane
        // its own entry i = q while q < j and, for q > j, its partner's entry
        // i = 31 - q, which a shuffle moves into the partner's ec[31 - q]:
        // sixteen entropy terms per lane instead of thirty-one.
        float ec[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) ec[i] = PINF;
        {
          const bool low = lane < 16;
          const int tp = t0 + 31 - lane;  // the partner's t (for low lanes)
          const bool pv = low && tp <= k;
          int tdp[TDW];
#pragma unroll
          for (int c = 0; c < TDW; ++c) tdp[c] = (pv && c < SW) ? sd[tp * SW + c] : 0;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const bool own = tv && q < lane;
            const bool part = pv && q > lane;
            int row[TDW];
#pragma unroll
            for (int c = 0; c < TDW; ++c) row[c] = own ? td[c] : tdp[c];
            float v = PINF;
            if (own || part) v = entropy_w<TDW>(Lt, sd, SW, yhat, row, own ? t0 + q : t0 + 31 - q);
            if (own) ec[q] = v;
            const float recv = __shfl_sync(0xffffffffu, v, 31 - lane);
            if (!low && tv && 31 - q < lane) ec[31 - q] = recv;
          }
        }
        float rcur = tv ? Rt[t * LS] : NINF;  // level 1
#pragma unroll
        for (int li = 0; li < LEV; ++li) {
          const int l = li + 2;
          if (l > lmax) break;
          float* rb = rbuf + (li & 1) * 32;
          rb[lane] = rcur;
          __syncwarp();
          float m0 = acc[li], m1 = NINF;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 r = reinterpret_cast<const float4*>(rb)[q];
            m0 = fmax3(m0, r.x - ec[4 * q + 0], r.y - ec[4 * q + 1]);
            m1 = fmax3(m1, r.z - ec[4 * q + 2], r.w - ec[4 * q + 3]);
          }
          const float v = fmaxf(m0, m1);
          if (tv) {
            if (l != lmax) Rt[t * LS + (l - 1)] = v;
            else if (t == k) *Rtop = v;  // the last level is read at t = k only
          }
          rcur = tv ? v : NINF;
        }
        __syncwarp();
      }

      // ---- traceback: l*(l) = the level of the largest R(k, l'), l' <= l
      // (the first in increasing l'), from one warp scan
      {
        float cbest = Rget(k, 1);
        int carg = 1;
        for (int l0 = 2; l0 <= lmax; l0 += 32) {
          const int l = l0 + lane;
          float v = l <= lmax ? Rget(k, l) : NINF;
          int a = l;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const float ov = __shfl_up_sync(0xffffffffu, v, d);
            const int oa = __shfl_up_sync(0xffffffffu, a, d);
            if (lane >= d && !(v > ov)) {
              v = ov;
              a = oa;
            }
          }
          if (!(v > cbest)) {
            v = cbest;
            a = carg;
          }
          if (l <= lmax) lst[l] = a;
          cbest = __shfl_sync(0xffffffffu, v, 31);
          carg = __shfl_sync(0xffffffffu, a, 31);
        }
      }
      __syncwarp();
      // one path per group of G lanes (at least 4, at most 8 groups), from
      // (k, l*) down: at (t, lv) the largest s with R(s, lv-1) - E(s, t)
      // equal to R(t, lv); then the path re-scored in double
      const int npaths = lmax - 1;
      int G = 32;
      while (G > 4 && 32 / G < npaths) --G;
      const int NG = 32 / G;
      const int grp = lane / G, sub = lane - grp * G;
      const unsigned gmask = G == 32 ? 0xffffffffu : (1u << G) - 1u;
      int* gcut = cuts + min(grp, 7) * S.xmax;
      for (int base = 0; base < npaths; base += NG) {
        const int pidx = base + grp;
        const bool act = grp < NG && pidx < npaths;
        const int l = lmax - pidx;
        const int lstar = act ? lst[l] : 1;
        int lv = lstar, tcur = k, s0 = k - 1;
        bool going = act && lv >= 2;
        float target = going ? Rget(k, lv) : NINF;
        int td[TDW];
#pragma unroll
        for (int c = 0; c < TDW; ++c) td[c] = c < SW ? sd[tcur * SW + c] : 0;
        while (__any_sync(0xffffffffu, going)) {
          const int s = s0 - sub;
          bool hit = false;
          if (going && s >= lv - 1) {
            const float r = Rt[s * LS + (lv - 2)];
            const float e = entropy_w<TDW>(Lt, sd, SW, yhat, td, s);
            hit = r >= target && r - e == target;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, hit);
          const unsigned m = grp < NG ? (bal >> (G * grp)) & gmask : 0u;
          if (going) {
            int found = -1;
            if (m) found = s0 - (__ffs(m) - 1);
            else if (s0 - G < lv - 1) found = lv - 1;  // unreachable: R(t,lv) is a candidate
            if (found >= 0) {
              if (sub == 0) gcut[lv - 2] = found;
              tcur = found;
              --lv;
              s0 = tcur - 1;
              if (lv >= 2) {
                target = Rget(tcur, lv);
#pragma unroll
                for (int c = 0; c < TDW; ++c) td[c] = c < SW ? sd[tcur * SW + c] : 0;
              } else {
                going = false;
              }
            } else {
              s0 -= G;
            }
          }
        }
        __syncwarp();
        // -E(0,s_1) - E(s_1,s_2) - ... - E(s_{l*-1},k) in double, the terms
        // (column c, row r) spread over the group's lanes
        double part = 0.0;
        if (act) {
          const int nt = lstar * (yhat + 1);
          for (int i = sub; i < nt; i += G) {
            const int c = i / (yhat + 1), r = i - c * (yhat + 1);
            const int a = c == 0 ? 0 : gcut[c - 1];
            const int bnd = c == lstar - 1 ? k : gcut[c];
            const double Lv = P.L64[sd[bnd * SW + r] - sd[a * SW + r]];
            part += r == 0 ? -Lv : Lv;
          }
        }
        double tot = part;
        for (int j = 1; j < G; ++j) {
          const double ov = __shfl_sync(0xffffffffu, part, min(lane + j, 31));
          if (sub + j < G) tot += ov;
        }
        if (act && sub == 0) Iw[l] = HQ + tot / (double)n;
        if (act && P.trace.d_cuts) {
          int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
          for (int c = sub; c < l - 1; c += G) dst[c] = c < lstar - 1 ? gcut[c] : k;
        }
        __syncwarp();
      }
      __syncwarp();
      if (lane == 0 && lmax >= 2) {
        // subtract-and-max candidates of the R recursion (as in k_dp.cuh)
        const long long Lm = lmax, K = k;
        long long cand = (Lm + 1) * Lm * (Lm - 1) / 6;
        const long long tsum = (K * (K + 1) - Lm * (Lm + 1)) / 2;
        cand += (Lm - 1) * tsum - (K - Lm) * (Lm - 1) * Lm / 2;
        cand_sum += cand;
      }
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
    if (lane == 0) {
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

namespace {

typedef void (*dp_warp_kernel_t)(DPParams, WarpPlan);

dp_warp_kernel_t dp_warp_pick(int lev, int tdw) {
  // 8 and 12 levels: above that the blocked CTA kernel (k_dp.cuh), whose
  // R table is shared by more warps, is faster
  if (tdw == 8) {
    switch (lev) {
      case 8: return k_dp_warp<8, 8>;
      case 12: return k_dp_warp<12, 8>;
      default: return nullptr;
    }
  }
  if (tdw == 16) {
    switch (lev) {
      case 8: return k_dp_warp<8, 16>;
      case 12: return k_dp_warp<12, 16>;
      default: return nullptr;
    }
  }
  return nullptr;
}

}  // namespace

bool dp_warp_supported(int lev, int tdw) { return dp_warp_pick(lev, tdw) != nullptr; }

cudaError_t dp_warp_configure(int lev, int tdw, int smem, int threads, int* blocks_per_sm,
                              bool set_attr) {
  const dp_warp_kernel_t k = dp_warp_pick(lev, tdw);
  if (!k) return cudaErrorInvalidValue;
  if (set_attr) {
    const cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k), smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t dp_warp_launch(int lev, int tdw, int grid, int threads, int smem, cudaStream_t st,
                           const DPParams& P, const WarpPlan& S) {
  const dp_warp_kernel_t k = dp_warp_pick(lev, tdw);
  if (!k) return cudaErrorInvalidValue;
  k<<<grid, threads, smem, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace gm
