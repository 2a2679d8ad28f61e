// k_dp.cuh -- the OptimizeXAxis dynamic program (SOM Algorithm 2 with the
// precomputations of Appendix item 10), one CTA per task, persistent over an
// atomic task queue.
//
// The DP over superclump ends c_0 < ... < c_k,
//   W(t,1) = -E(0,t),  W(t,l) = max_{s in [l-1, t]} W(s,l-1) - E(s,t),
// (s = t is an empty last column, E(t,t) = 0) is computed through the
// recursion without empty columns,
//   R(t,1) = -E(0,t),  R(t,l) = max_{s in [l-1, t-1]} R(s,l-1) - E(s,t),
// and W(t,l) = max_{l' <= l} R(t,l').  The two give the same doubles: each
// W(s,l-1) is one of the R(s,l'') (a maximum picks one of its arguments),
// and rounding is monotone, so W(s,l-1) - E(s,t) is the largest of the
// R(s,l'') - E(s,t), each of which is a candidate of some R(t,l''+1).  The
// maximum needs no argument; the chosen partitions are recovered afterwards
// by a traceback.
//
// Schedule.  t runs in blocks of 32; lane j of every warp owns t = t0 + j.
// For block b+1 the candidates split into
//   A1: s below block b  (rows final before block b is solved),
//   A2: s inside block b (rows final once block b is solved),
//   B:  s inside block b+1 itself, one t after another.
// Warp 0 solves block b (its part B) while the other warps work through A1
// of block b+1, taking s-chunks from a shared counter (warp 0 joins when it
// is done); then all warps do A2.  In A1/A2 each lane computes E(s,t) once
// and updates the running maxima of a group of levels with R(s,l-1) - E
// (the R row is a warp-wide 16-byte broadcast); the warps' partial maxima
// meet in shared memory through atomicMin on the value bits (every value is
// -0.0, negative or -inf, so a larger value has smaller bits).  Levels
// beyond a task's last level hold -inf, so no candidate needs a guard.
#pragma once
#include <type_traits>

#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

template <typename real>
struct Bits;
template <>
struct Bits<float> {
  using U = unsigned int;
  __device__ static U of(float v) { return __float_as_uint(v); }
  __device__ static float from(U b) { return __uint_as_float(b); }
  __device__ static float ninf() { return __int_as_float(0xff800000); }
  __device__ static float max(float a, float b) { return fmaxf(a, b); }
};
template <>
struct Bits<double> {
  using U = unsigned long long;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
  __device__ static double from(U b) { return __longlong_as_double((long long)b); }
  __device__ static double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
  __device__ static double max(double a, double b) { return fmax(a, b); }
};

// E(s,t) = L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s]), increasing r
template <typename real>
__device__ __forceinline__ real entropy_term(const real* __restrict__ Lt, const int* __restrict__ scb,
                                             const int* __restrict__ cum, int ks, int yhat, int s,
                                             int t) {
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

__device__ __forceinline__ double entropy_term64g(const double* __restrict__ L64,
                                                  const int* __restrict__ scb,
                                                  const int* __restrict__ cum, int ks, int yhat,
                                                  int s, int t) {
  double e = L64[scb[t] - scb[s]];
  const int* __restrict__ ct = cum + t;
  const int* __restrict__ cs = cum + s;
  int r = 0;
  // four rows at a time: the loads run ahead, the subtractions keep the
  // order of increasing r
  for (; r + 4 <= yhat; r += 4) {
    const double l0 = L64[ct[(r + 0) * ks] - cs[(r + 0) * ks]];
    const double l1 = L64[ct[(r + 1) * ks] - cs[(r + 1) * ks]];
    const double l2 = L64[ct[(r + 2) * ks] - cs[(r + 2) * ks]];
    const double l3 = L64[ct[(r + 3) * ks] - cs[(r + 3) * ks]];
    e -= l0;
    e -= l1;
    e -= l2;
    e -= l3;
  }
  for (; r < yhat; ++r) e -= L64[ct[r * ks] - cs[r * ks]];
  return e;
}

// Candidates R(s, l-1) - E(s, t) for s in [s_lo, s_hi] and the LEV levels
// l = lc .. lc+LEV-1 (R columns lc-2 ..), max-accumulated into acc.
template <typename real, int LEV>
__device__ __forceinline__ void accumulate(real (&acc)[LEV], const real* __restrict__ Rt, int LS,
                                           int lc, int s_lo, int s_hi, const real* __restrict__ Lt,
                                           const int* __restrict__ scb, const int* __restrict__ cum,
                                           int ks, int yhat, int tt) {
  using BT = Bits<real>;
  constexpr int VW = 16 / sizeof(real);
  // E(s+1, t) is computed while the candidates of s are formed
  real e = entropy_term<real>(Lt, scb, cum, ks, yhat, s_lo, tt);
#pragma unroll 1
  for (int s = s_lo; s <= s_hi; ++s) {
    const real en = s < s_hi ? entropy_term<real>(Lt, scb, cum, ks, yhat, s + 1, tt) : e;
    const real* Rs = Rt + s * LS + (lc - 2);
#pragma unroll
    for (int g = 0; g < LEV / VW; ++g) {
      if constexpr (sizeof(real) == 4) {
        const float4 r = *reinterpret_cast<const float4*>(Rs + 4 * g);
        acc[4 * g + 0] = BT::max(acc[4 * g + 0], r.x - e);
        acc[4 * g + 1] = BT::max(acc[4 * g + 1], r.y - e);
        acc[4 * g + 2] = BT::max(acc[4 * g + 2], r.z - e);
        acc[4 * g + 3] = BT::max(acc[4 * g + 3], r.w - e);
      } else {
        const double2 r = *reinterpret_cast<const double2*>(Rs + 2 * g);
        acc[2 * g + 0] = BT::max(acc[2 * g + 0], r.x - e);
        acc[2 * g + 1] = BT::max(acc[2 * g + 1], r.y - e);
      }
    }
    e = en;
  }
}

template <typename real, int LEV>
__device__ __forceinline__ void flush(const real (&acc)[LEV], typename Bits<real>::U* Xrow, int lc,
                                      int lmax) {
  using BT = Bits<real>;
#pragma unroll
  for (int i = 0; i < LEV; ++i)
    if (lc + i <= lmax) atomicMin(&Xrow[lc + i - 1], BT::of(acc[i]));
}

// Phase A over the s range [s_begin, s_end) of one part (A1 with a shared
// work counter, or A2 with a static split), LEV levels per pass.
template <typename real, int LEV>
__device__ __forceinline__ void phase_a(const real* __restrict__ Rt, int LS, int lmax, int s_begin, int s_end,
                        bool stealing, int* s_next, const real* __restrict__ Lt,
                        const int* __restrict__ scb, const int* __restrict__ cum, int ks, int yhat,
                        int tt, bool tv, typename Bits<real>::U* Xrow, int warp, int NW, int lane) {
  using BT = Bits<real>;
  const int CH = stealing ? 8 : 4;  // s per grab
  const int nlev = lmax - 1;
  const int npass = (nlev + LEV - 1) / LEV;
  const int nsb = (s_end - s_begin + CH - 1) / CH;  // s-chunks per pass
  if (nsb <= 0) return;
  real acc[LEV];
  int cur_pass = -1;
  int g = stealing ? 0 : warp;
  for (;;) {
    if (stealing) {
      int gg = 0;
      if (lane == 0) gg = atomicAdd(s_next, 1);
      g = __shfl_sync(0xffffffffu, gg, 0);
    }
    if (g >= nsb * npass) break;
    const int pass = g / nsb;
    const int sb = g - pass * nsb;
    if (pass != cur_pass) {
      if (cur_pass >= 0 && tv) flush<real, LEV>(acc, Xrow, 2 + cur_pass * LEV, lmax);
#pragma unroll
      for (int i = 0; i < LEV; ++i) acc[i] = BT::ninf();
      cur_pass = pass;
    }
    const int s_lo = s_begin + sb * CH;
    const int s_hi = min(s_end - 1, s_lo + CH - 1);
    accumulate<real, LEV>(acc, Rt, LS, 2 + pass * LEV, s_lo, s_hi, Lt, scb, cum, ks, yhat, tt);
    if (!stealing) g += NW;
  }
  if (cur_pass >= 0 && tv) flush<real, LEV>(acc, Xrow, 2 + cur_pass * LEV, lmax);
}

__host__ __device__ __forceinline__ int level_group(int nlev) {
  if (nlev <= 4) return 4;
  if (nlev <= 8) return 8;
  if (nlev <= 12) return 12;
  if (nlev <= 16) return 16;
  if (nlev <= 20) return 20;
  if (nlev <= 24) return 24;
  if (nlev <= 32) return 32;
  return 40;
}

// The candidates of block b with s inside the block, one t after another,
// with the block's earlier rows kept in registers (at most 32 levels, level
// 2 + lane in lane `lane`): right after step i, the lane of level l receives
// R(t0+i, l-1) from the lane of level l-1 by one shuffle, so step j reads
// registers and the broadcast E column only.  The 32 steps are unrolled so
// that every register index is static.
template <typename real>
__device__ __forceinline__ void phase_b_regs(real* __restrict__ Rt, real* __restrict__ Rtop, int LS,
                                             int LX, int lmax, int t0, int k,
                                             const typename Bits<real>::U* __restrict__ Xcur,
                                             bool has_x, const real* __restrict__ Eb, int lane) {
  using BT = Bits<real>;
  const int l = 2 + lane;
  const bool live = l <= lmax;
  real prev[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (t0 + j > k) break;
    const int tj = t0 + j;
    real v = (has_x && live) ? BT::from(Xcur[j * LX + (l - 1)]) : BT::ninf();
#pragma unroll
    for (int i = 0; i < j; ++i) v = BT::max(v, prev[i] - Eb[i * 33 + j]);
    if (live) {
      if (l == lmax) Rtop[tj] = v; else Rt[tj * LS + (l - 1)] = v;
    }
    const real below = __shfl_sync(0xffffffffu, v, (lane + 31) & 31);
    prev[j] = lane == 0 ? Rt[tj * LS] : below;
  }
}

template <typename real, bool RSM, int LEV>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 2 : 1)
k_dp(DPParams P, DPPlan S) {
  using BT = Bits<real>;
  using U = typename BT::U;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_task;
  __shared__ int s_next;
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int NW = T >> 5;
  constexpr bool fp32 = sizeof(real) == 4;

  // R table [kmax+1][LS]: R(t, l) at column l-1 for the source levels
  // l = 1..lmax-1 (row s = 0 at -inf); the last level lmax in Rtop[t].
  // Shared memory (RSM) or, for very large B, global memory.
  real* Rt = RSM ? reinterpret_cast<real*>(sm + S.off_R)
                 : reinterpret_cast<real*>(P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta);
  real* Rtop = reinterpret_cast<real*>(sm + S.off_Rtop);  // [kmax+1]
  U* Xb = reinterpret_cast<U*>(sm + S.off_X);             // [2][32][LX] bits
  real* Eb = reinterpret_cast<real*>(sm + S.off_Eb);      // [32][33]
  int* scb = reinterpret_cast<int*>(sm + S.off_scb);      // [kmax+1]
  int* cum = reinterpret_cast<int*>(sm + S.off_cum);      // [cum_max]
  // after the DP the X buffers hold the traceback scratch
  int* cuts = reinterpret_cast<int*>(sm + S.off_X);                       // [NW][xmax]
  double* Iw = reinterpret_cast<double*>(sm + S.off_X + S.off_I_rel);     // [xmax+1]
  double* Ecw = reinterpret_cast<double*>(sm + S.off_X + S.off_ecol_rel);  // [NW][xmax+1]
  const int LS = S.LS;
  const int LX = S.LX;
  const real* Lt;  // L(m) = m ln m, m = 0..n
  {
    const real* Lsrc;
    if constexpr (fp32) Lsrc = P.L32; else Lsrc = P.L64;
    if constexpr (RSM) {
      real* Ls = reinterpret_cast<real*>(sm + S.off_L);
      for (int m = tid; m <= P.n_full; m += T) Ls[m] = Lsrc[m];
      Lt = Ls;
    } else {
      Lt = Lsrc;
    }
  }
  const real NINF = BT::ninf();
  const U NINF_BITS = BT::of(NINF);
  const int64_t C = P.chunk_pairs;

  for (;;) {
    if (tid == 0) s_task = (long long)atomicAdd(P.queue, 1ull) + P.task_begin;
    __syncthreads();
    const int64_t task = s_task;
    __syncthreads();
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
    if (tid == 0 && P.trace.d_k) {
      P.trace.d_k[trace_task] = k;
      if (P.trace.d_yhat) P.trace.d_yhat[trace_task] = yhat;
      if (P.trace.d_clumps) P.trace.d_clumps[trace_task] = valid ? rec[2] : 0;
    }
    if (!valid) continue;
    const double HQ = *reinterpret_cast<const double*>(rec + 4);
    const int x = B / y;
    const int ks = k + 1;
    const int lmax = min(x, k);
    for (int j = tid; j <= k; j += T) scb[j] = rec[6 + j];
    for (int i = tid; i < yhat * ks; i += T) cum[i] = rec[6 + ks + i];
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = tid; j <= k; j += T) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncthreads();
    // R(t, l) for 1 <= l <= lmax
    auto Rget = [&](int t, int l) -> real { return l == lmax ? Rtop[t] : Rt[t * LS + (l - 1)]; };

    if (k >= 2) {
      for (int i = tid; i < ks * LS; i += T) Rt[i] = NINF;
      for (int i = tid; i < ks; i += T) Rtop[i] = NINF;
      for (int i = tid; i < 2 * 32 * LX; i += T) Xb[i] = NINF_BITS;
      __syncthreads();
      for (int t = 1 + tid; t <= k; t += T) {
        const real r1 = -entropy_term<real>(Lt, scb, cum, ks, yhat, 0, t);
        if (lmax == 1) Rtop[t] = r1; else Rt[t * LS] = r1;
      }
      for (int idx = tid; idx < 32 * 32; idx += T) {  // within-block entropies of block 0
        const int i = idx >> 5, j = idx & 31;
        if (i < j && 1 + j <= k) Eb[i * 33 + j] = entropy_term<real>(Lt, scb, cum, ks, yhat, 1 + i, 1 + j);
      }
      if (tid == 0) s_next = 0;
      __syncthreads();

      const int nb = (k + 31) / 32;
      for (int b = 0; b < nb; ++b) {
        const int t0 = 1 + 32 * b;
        const int t1 = t0 + 32;  // first t of block b+1
        const bool next = t1 <= k;
        U* Xcur = Xb + (b & 1) * 32 * LX;
        U* Xnxt = Xb + ((b + 1) & 1) * 32 * LX;
        const int tn = t1 + lane;  // this lane's t in block b+1
        const bool tnv = next && tn <= k;
        const int ttn = tnv ? tn : k;
        for (int step = 0; step < 2; ++step) {
          if (step == 0 && warp == 0) {
            // ---- block b, s inside the block: one t after another
            if (std::is_same<real, float>::value && LEV <= 24 && lmax - 1 <= 32) {
              phase_b_regs<real>(Rt, Rtop, LS, LX, lmax, t0, k, Xcur, b > 0, Eb, lane);
            } else {
              // many levels: lanes over levels, two per lane per pass
              for (int j = 0; j < 32 && t0 + j <= k; ++j) {
                const int tj = t0 + j;
                for (int lb = 2; lb <= lmax; lb += 64) {
                  const int la = lb + lane, lc2 = lb + 32 + lane;
                  const bool va = la <= lmax, vb = lc2 <= lmax;
                  real a0 = NINF, a1 = NINF, b0 = NINF, b1 = NINF;
                  if (b > 0) {
                    if (va) a0 = BT::from(Xcur[j * LX + (la - 1)]);
                    if (vb) b0 = BT::from(Xcur[j * LX + (lc2 - 1)]);
                  }
                  const real* Ra = Rt + t0 * LS + (la - 2);
                  const real* Rb = Rt + t0 * LS + (lc2 - 2);
                  int i = 0;
                  for (; i + 1 < j; i += 2) {
                    const real e0 = Eb[i * 33 + j], e1 = Eb[(i + 1) * 33 + j];
                    if (va) {
                      a0 = BT::max(a0, Ra[i * LS] - e0);
                      a1 = BT::max(a1, Ra[(i + 1) * LS] - e1);
                    }
                    if (vb) {
                      b0 = BT::max(b0, Rb[i * LS] - e0);
                      b1 = BT::max(b1, Rb[(i + 1) * LS] - e1);
                    }
                  }
                  if (i < j) {
                    const real e0 = Eb[i * 33 + j];
                    if (va) a0 = BT::max(a0, Ra[i * LS] - e0);
                    if (vb) b0 = BT::max(b0, Rb[i * LS] - e0);
                  }
                  if (va) {
                    const real v = BT::max(a0, a1);
                    if (la == lmax) Rtop[tj] = v; else Rt[tj * LS + (la - 1)] = v;
                  }
                  if (vb) {
                    const real v = BT::max(b0, b1);
                    if (lc2 == lmax) Rtop[tj] = v; else Rt[tj * LS + (lc2 - 1)] = v;
                  }
                }
                __syncwarp();
              }
            }
          }
          // step 0: A1 of block b+1, s in [1, t0 - 1], shared work counter
          // (warp 0 joins once block b is solved);
          // step 1: A2 of block b+1, s in block b, static split
          const bool stealing = step == 0;
          const int sb0 = stealing ? 1 : t0;
          const int sb1 = stealing ? t0 : t1;
          if (next && sb1 > sb0)
            phase_a<real, LEV>(Rt, LS, lmax, sb0, sb1, stealing, &s_next, Lt, scb, cum, ks, yhat, ttn,
                               tnv, Xnxt + lane * LX, warp, NW, lane);
          if (step == 1) {
            for (int i = tid; i < 32 * LX; i += T) Xcur[i] = NINF_BITS;  // for block b+2
            if (tid == 0) s_next = 0;
            if (next)
              for (int idx = tid; idx < 32 * 32; idx += T) {  // within-block entropies of block b+1
                const int i = idx >> 5, j = idx & 31;
                if (i < j && t1 + j <= k)
                  Eb[i * 33 + j] = entropy_term<real>(Lt, scb, cum, ks, yhat, t1 + i, t1 + j);
              }
          }
          __syncthreads();
        }
      }
    }

    // ---- I(l) for l = 2..x
    const bool need_paths = fp32 || P.trace.d_cuts != nullptr;
    if (k >= 2 && need_paths) {
      int* mycut = cuts + warp * S.xmax;
      if constexpr (fp32) {
        // Traceback in the R recursion: l* = the level of the largest R(k, l'),
        // l' <= l (first in increasing l'), then at (t, lv) an s with
        // R(s, lv-1) - E(s, t) equal to R(t, lv) (an exact match exists: a
        // maximum is one of its candidates).  The scan runs down from t - 1,
        // so it covers about one column; since E >= 0, an s with R(s, lv-1)
        // below the target cannot match and its E is not formed.
        for (int l = 2 + warp; l <= lmax; l += NW) {
          int lstar = 1;
          real best = Rget(k, 1);
          for (int lv = 2; lv <= l; ++lv) {
            const real r = Rget(k, lv);
            if (r > best) {
              best = r;
              lstar = lv;
            }
          }
          int tcur = k;
          for (int lv = lstar; lv >= 2; --lv) {
            const real target = Rget(tcur, lv);
            int found = -1;
            for (int s0 = tcur - 1; s0 >= lv - 1 && found < 0; s0 -= 32) {
              const int s = s0 - lane;
              bool hit = false;
              if (s >= lv - 1) {
                const real r = Rt[s * LS + (lv - 2)];
                if (r >= target) hit = r - entropy_term<real>(Lt, scb, cum, ks, yhat, s, tcur) == target;
              }
              const unsigned m = __ballot_sync(0xffffffffu, hit);
              if (m) found = s0 - (__ffs(m) - 1);
            }
            if (found < 0) found = lv - 1;  // unreachable: R(t,lv) is one of its candidates
            if (lane == 0) mycut[lv - 2] = found;
            tcur = found;
          }
          __syncwarp();
          // re-score the chosen partition in double, in the DP's own order:
          // w = -E(0,s_1) - E(s_1,s_2) - ... - E(s_{l*-1},k)
          double* ec = Ecw + warp * (S.xmax + 1);
          for (int c = lane; c < lstar; c += 32) {
            const int a = c == 0 ? 0 : mycut[c - 1];
            const int bnd = c == lstar - 1 ? k : mycut[c];
            ec[c] = entropy_term64g(P.L64, scb, cum, ks, yhat, a, bnd);
          }
          __syncwarp();
          double w = -ec[0];
          for (int c = 1; c < lstar; ++c) w = w - ec[c];
          if (lane == 0) Iw[l] = HQ + w / (double)n;
          if (P.trace.d_cuts) {
            // as l - 1 column ends: the l* - 1 cuts, then empty columns at k
            int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
            for (int c = lane; c < l - 1; c += 32) dst[c] = c < lstar - 1 ? mycut[c] : k;
          }
          __syncwarp();
        }
      } else {
        // W = prefix maximum of R over levels (in place), then the oracle's
        // rule: at (t, lv) the first s in [lv-1, t] maximising W(s,lv-1) -
        // E(s,t), s = t being an empty column.
        for (int s = 1 + tid; s <= k; s += T) {
          real wv = Rt[s * LS];
          for (int l = 2; l < lmax; ++l) {
            wv = BT::max(wv, Rt[s * LS + (l - 1)]);
            Rt[s * LS + (l - 1)] = wv;
          }
          Rtop[s] = BT::max(wv, Rtop[s]);
        }
        __syncthreads();
        for (int l = 2 + warp; l <= lmax; l += NW) {
          int tcur = k;
          for (int lv = l; lv >= 2; --lv) {
            real best = NINF;
            int arg = 0x7fffffff;
            for (int s = lv - 1 + lane; s <= tcur; s += 32) {
              const real wv = Rt[s * LS + (lv - 2)];
              const real cand = (s == tcur) ? wv : wv - entropy_term<real>(Lt, scb, cum, ks, yhat, s, tcur);
              if (cand > best) {
                best = cand;
                arg = s;
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
            if (lane == 0) mycut[lv - 2] = arg;
            tcur = arg;
          }
          __syncwarp();
          if (lane == 0) Iw[l] = HQ + (double)Rget(k, l) / (double)n;
          if (P.trace.d_cuts) {
            int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
            for (int c = lane; c < l - 1; c += 32) dst[c] = mycut[c];
          }
          __syncwarp();
        }
      }
      __syncthreads();
    }

    const int rowoff = row_offset(B, y);
    double* Mo = P.Mo + ((int64_t)pl * 2 + o) * P.cells_max + rowoff;
    for (int l = 2 + tid; l <= x; l += T) {
      double I;
      if (k <= 1) {
        I = 0.0;
      } else if (need_paths) {
        I = Iw[min(l, k)];
      } else {
        const int lc = min(l, k);
        real w = Rget(k, 1);
        for (int lv = 2; lv <= lc; ++lv) w = BT::max(w, Rget(k, lv));
        I = HQ + (double)w / (double)n;
      }
      const int mn = min(l, yhat);
      Mo[l - 2] = mn < 2 ? 0.0 : I / P.lnt[mn];
      if (P.trace.d_I) P.trace.d_I[trace_task * P.trace.I_stride + (l - 2)] = I;
      if (P.trace.d_cuts && (l > k || k <= 1)) {
        int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
        for (int c = 0; c < l - 1; ++c) dst[c] = -1;
      }
    }
    if (tid == 0 && yhat < 2) atomicOr(&P.pp.flags[pl], 1 << GMINE_E_CONSTANT);
    if (tid == 0 && P.counters) {
      // subtract-and-max candidates of the R recursion:
      // sum_{t=2}^{k} sum_{l=2}^{min(t,lmax)} (t - l + 1)
      //   = C(lmax+1, 3) + (lmax-1) * sum_{t=lmax+1}^{k} (t - lmax/2)
      long long cand = 0;
      if (k >= 2 && lmax >= 2) {
        const long long L = lmax, K = k;
        cand = (L + 1) * L * (L - 1) / 6;
        const long long tsum = (K * (K + 1) - L * (L + 1)) / 2;
        cand += (L - 1) * tsum - (K - L) * (L - 1) * L / 2;
      }
      atomicAdd(reinterpret_cast<unsigned long long*>(P.counters), (unsigned long long)cand);
      atomicAdd(reinterpret_cast<unsigned long long*>(P.counters) + 1, 1ull);
    }
    __syncthreads();
  }
}

typedef void (*dp_kernel_t)(DPParams, DPPlan);

// Per-translation-unit wrappers: each of k_dp_{f32,f64}_{smem,global}.cu
// instantiates the kernel for one precision and one placement of the R
// table and defines these two functions for it (so that every launch of a
// template instance happens in the unit that instantiates it).
#define GM_DP_WRAPPERS(REAL, RSM, NAME, ...)                                               \
  static dp_kernel_t NAME##_pick(int lev) {                                              \
    switch (lev) {                                                                       \
      __VA_ARGS__                                                                        \
    }                                                                                    \
  }                                                                                      \
  cudaError_t NAME##_configure(int lev, int smem, int threads, int* blocks_per_sm) {     \
    const dp_kernel_t k = NAME##_pick(lev);                                              \
    const cudaError_t e =                                                                \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);     \
    if (e != cudaSuccess) return e;                                                      \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem); \
  }                                                                                      \
  cudaError_t NAME##_launch(int lev, int grid, int threads, int smem, cudaStream_t st,    \
                            const DPParams& P, const DPPlan& S) {                        \
    NAME##_pick(lev)<<<grid, threads, smem, st>>>(P, S);                                 \
    return cudaGetLastError();                                                           \
  }

}  // namespace gm
