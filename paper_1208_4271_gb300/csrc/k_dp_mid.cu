// k_dp_mid.cu -- the OptimizeXAxis dynamic program (SOM Algorithm 2 with the
// precomputations of Appendix item 10), one CTA per task, level after level,
// for tasks whose whole entropy triangle fits in shared memory.
//
// The recursion is the one of k_dp.cuh without empty columns,
//   R(t,1) = -E(0,t),  R(t,l) = max_{s in [l-1, t-1]} R(s,l-1) - E(s,t),
// whose prefix maximum over levels is the method's W(t,l) exactly.  Within a
// level every t is independent, so the only sequential chain is the levels
// (x - 1 of them) instead of the superclumps (k of them).  E(s,t) for all
// s < t (Appendix item 10b: the entropy matrix) is formed once, warps over
// rows s and lanes over t.  Each level below the last then runs over tiles
// of 32 t (lanes) by 32 s dealt round-robin to the warps: the R row entry is
// a warp-wide broadcast, E(s, t..t+31) 32 consecutive words, and the tile's
// maxima join the level row through atomicMin on the value bits (every
// value is -0.0, negative or -inf, so a larger value has smaller bits).  The
// last level is needed at t = k only (W(k,l) and the tracebacks never read
// it elsewhere): one CTA-wide maximum.
#include "gmine_internal.cuh"
#include "kernels.h"

namespace gm {

template <typename real>
struct MBits;
template <>
struct MBits<float> {
  using U = unsigned int;
  __device__ static U of(float v) { return __float_as_uint(v); }
  __device__ static float from(U b) { return __uint_as_float(b); }
  __device__ static float ninf() { return __int_as_float(0xff800000); }
  __device__ static float max(float a, float b) { return fmaxf(a, b); }
};
// The values compared here (R, its candidates R - E with E >= +0, -inf)
// lie in [-inf, -0.0], where the order of doubles is the reverse of the
// order of their bit patterns: the maximum is an integer minimum, on the
// integer pipe instead of GB300's two FP64 operations per clock and SM.
template <>
struct MBits<double> {
  using U = unsigned long long;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
  __device__ static double from(U b) { return __longlong_as_double((long long)b); }
  __device__ static double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
  __device__ static double max(double a, double b) {
    const U x = of(a), y = of(b);
    return from(y < x ? y : x);
  }
};

__device__ __forceinline__ float mid_max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ double mid_max3(double a, double b, double c) {
  return MBits<double>::max(MBits<double>::max(a, b), c);  // values in [-inf, -0.0]
}

// E(s,t) = L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s]), increasing r
template <typename real>
__device__ __forceinline__ real entropy_mid(const real* __restrict__ Lt, const int* __restrict__ scb,
                                            const int* __restrict__ cum, int ks, int yhat, int s,
                                            int t) {
  real e = Lt[scb[t] - scb[s]];
  const int* __restrict__ ct = cum + t;
  const int* __restrict__ cs = cum + s;
  int r = 0;
  for (; r + 4 <= yhat; r += 4) {  // loads ahead, subtractions in increasing r
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

// E(s,t1) and E(s,t2) with their loads interleaved (two independent chains,
// each in increasing r)
template <typename real>
__device__ __forceinline__ void entropy_mid2(const real* __restrict__ Lt, const int* __restrict__ scb,
                                             const int* __restrict__ cum, int ks, int yhat, int s,
                                             int t1, int t2, real& e1, real& e2) {
  real a = Lt[scb[t1] - scb[s]];
  real b = Lt[scb[t2] - scb[s]];
  const int* __restrict__ cs = cum + s;
  const int* __restrict__ c1 = cum + t1;
  const int* __restrict__ c2 = cum + t2;
  int r = 0;
  for (; r + 4 <= yhat; r += 4) {
    real la[4], lb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = cs[(r + q) * ks];
      la[q] = Lt[c1[(r + q) * ks] - v];
      lb[q] = Lt[c2[(r + q) * ks] - v];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a -= la[q];
      b -= lb[q];
    }
  }
  for (; r < yhat; ++r) {
    const int v = cs[r * ks];
    a -= Lt[c1[r * ks] - v];
    b -= Lt[c2[r * ks] - v];
  }
  e1 = a;
  e2 = b;
}

// offset of E(s, .) in the packed triangle: row s holds t = s+1 .. k
__device__ __forceinline__ int tri_row(int s, int k) { return s * k - (s * (s - 1)) / 2; }

template <typename real>
__global__ void __launch_bounds__(256) k_dp_mid(DPParams P, MidPlan S) {
  using BT = MBits<real>;
  using U = typename BT::U;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_task;
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int NW = T >> 5;
  constexpr bool fp32 = sizeof(real) == 4;

  real* Et = reinterpret_cast<real*>(sm + S.off_E);      // packed triangle
  real* Rl = reinterpret_cast<real*>(sm + S.off_R);      // [lmax+1][KS]: R(t,l) at l*KS+t
  real* Lt = reinterpret_cast<real*>(sm + S.off_L);      // [n+1]
  int* recb = reinterpret_cast<int*>(sm + S.off_rec);    // the task's record
  double* Iw = reinterpret_cast<double*>(sm + S.off_I);  // [xmax+1]
  int* cuts = reinterpret_cast<int*>(sm + S.off_cuts);   // [NW][xmax]
  double* Ecw = reinterpret_cast<double*>(sm + S.off_ecol);  // [NW][xmax+1]
  const int KS = S.KS;
  {
    const real* Lsrc;
    if constexpr (fp32) Lsrc = P.L32; else Lsrc = P.L64;
    for (int m = tid; m <= P.n_full; m += T) Lt[m] = Lsrc[m];
  }
  const real NINF = BT::ninf();
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
                         P.rec_off[y];
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
    copy_record(recb, rec, 6 + ks + yhat * ks, tid, T);
    const int* scb = recb + 6;      // superclump ends
    const int* cum = recb + 6 + ks;  // cum[r][t] at r * ks + t
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = tid; j <= k; j += T) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncthreads();

    if (k >= 2) {
      // ---- the entropy triangle: warps over rows s, lanes over t = s+1..k,
      // two entries per lane in flight
      for (int s = warp; s < k; s += NW) {
        real* row = Et + tri_row(s, k) - s - 1;  // row[t] = E(s,t)
        for (int t = s + 1 + lane; t <= k; t += 64) {
          const bool two = t + 32 <= k;
          real e1, e2;
          entropy_mid2<real>(Lt, scb, cum, ks, yhat, s, t, two ? t + 32 : t, e1, e2);
          row[t] = e1;
          if (two) row[t + 32] = e2;
        }
      }
      // level 1; every other level starts at -inf
      for (int i = tid; i < (lmax + 1) * KS; i += T) Rl[i] = NINF;
      __syncthreads();
      for (int t = 1 + tid; t <= k; t += T) Rl[KS + t] = -Et[tri_row(0, k) + t - 1];
      __syncthreads();
      // ---- levels 2 .. lmax-1 at every t >= l: tiles of 32 t (lanes) by
      // 32 s, the non-empty ones (some s < t) dealt round-robin to the
      // warps; a tile's maxima join the level row through atomicMin on the
      // value bits (distinct t per lane: no bank conflicts)
      for (int l = 2; l < lmax; ++l) {
        const real* Rp = Rl + (l - 1) * KS;
        U* Rc = reinterpret_cast<U*>(Rl + l * KS);
        const int nt = (k - l + 1 + 31) / 32;  // t-chunks [l + 32 i, l + 32 i + 31]
        // t-chunk i has s-pieces j = 0..i (s in [l-1 + 32 j, l + 32 j + 30]):
        // tile g = i (i + 1) / 2 + j
        const int ntiles = nt * (nt + 1) / 2;
        for (int g = warp; g < ntiles; g += NW) {
          int i = (int)((sqrtf(8.0f * (float)g + 1.0f) - 1.0f) * 0.5f);
          while (i * (i + 1) / 2 > g) --i;
          while ((i + 1) * (i + 2) / 2 <= g) ++i;
          const int j = g - i * (i + 1) / 2;
          const int t = l + 32 * i + lane;
          const int tt = min(t, k);
          const int sb = l - 1 + 32 * j;
          const int se = min(sb + 32, min(l + 32 * i + 31, k));  // s < the chunk's largest t
          real acc = NINF;
          int base = tri_row(sb, k) + tt - sb - 1;  // E(sb, tt); row s+1 starts k-s-1 later
          if (j < i) {
            // every s of the tile is below every t: two s per three-operand max
            int s = sb;
#pragma unroll 2
            for (; s + 1 < se; s += 2) {
              const int b1 = base + k - s - 1;
              acc = mid_max3(acc, Rp[s] - Et[base], Rp[s + 1] - Et[b1]);
              base = b1 + k - s - 2;
            }
            if (s < se) acc = BT::max(acc, Rp[s] - Et[base]);
          } else {
#pragma unroll 4
            for (int s = sb; s < se; ++s) {
              const real v = Rp[s] - Et[base];
              if (s < t) acc = BT::max(acc, v);
              base += k - s - 1;
            }
          }
          if (t <= k && acc != NINF) atomicMin(&Rc[t], BT::of(acc));
        }
        __syncthreads();
      }
      // ---- the last level at t = k only: R(k, lmax) over s in [lmax-1, k-1]
      {
        const int l = lmax;
        const real* Rp = Rl + (l - 1) * KS;
        real acc = NINF;
        for (int s = l - 1 + tid; s < k; s += T) acc = BT::max(acc, Rp[s] - Et[tri_row(s, k) + k - s - 1]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc = BT::max(acc, __shfl_xor_sync(0xffffffffu, acc, d));
        if (lane == 0 && acc != NINF) atomicMin(reinterpret_cast<U*>(Rl + l * KS) + k, BT::of(acc));
      }
      __syncthreads();
    }

    // ---- I(l) for l = 2..x
    const bool need_paths = fp32 || P.trace.d_cuts != nullptr;
    if (k >= 2 && need_paths) {
      int* mycut = cuts + warp * S.xmax;
      if constexpr (fp32) {
        // Traceback in the R recursion (as in k_dp.cu): l* = the level of the
        // largest R(k, l'), l' <= l; then at (t, lv) an s with R(s, lv-1) -
        // E(s, t) equal to R(t, lv), scanning down from t - 1.
        for (int l = 2 + warp; l <= lmax; l += NW) {
          int lstar = 1;
          real best = Rl[KS + k];
          for (int lv = 2; lv <= l; ++lv) {
            const real r = Rl[lv * KS + k];
            if (r > best) {
              best = r;
              lstar = lv;
            }
          }
          int tcur = k;
          for (int lv = lstar; lv >= 2; --lv) {
            const real target = Rl[lv * KS + tcur];
            int found = -1;
            for (int s0 = tcur - 1; s0 >= lv - 1 && found < 0; s0 -= 32) {
              const int s = s0 - lane;
              bool hit = false;
              if (s >= lv - 1) hit = Rl[(lv - 1) * KS + s] - Et[tri_row(s, k) + tcur - s - 1] == target;
              const unsigned m = __ballot_sync(0xffffffffu, hit);
              if (m) found = s0 - (__ffs(m) - 1);
            }
            if (found < 0) found = lv - 1;  // unreachable: R(t,lv) is one of its candidates
            if (lane == 0) mycut[lv - 2] = found;
            tcur = found;
          }
          __syncwarp();
          // re-score the chosen partition in double, in the DP's own order
          double* ec = Ecw + warp * (S.xmax + 1);
          for (int c = lane; c < lstar; c += 32) {
            const int a = c == 0 ? 0 : mycut[c - 1];
            const int bnd = c == lstar - 1 ? k : mycut[c];
            double e = P.L64[scb[bnd] - scb[a]];
            for (int r = 0; r < yhat; ++r) e -= P.L64[cum[r * ks + bnd] - cum[r * ks + a]];
            ec[c] = e;
          }
          __syncwarp();
          double w = -ec[0];
          for (int c = 1; c < lstar; ++c) w = w - ec[c];
          if (lane == 0) Iw[l] = HQ + w / (double)n;
          if (P.trace.d_cuts) {
            int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
            for (int c = lane; c < l - 1; c += 32) dst[c] = c < lstar - 1 ? mycut[c] : k;
          }
          __syncwarp();
        }
      } else {
        // W = prefix maximum of R over levels, then the method's rule: at
        // (t, lv) the first s in [lv-1, t] maximising W(s,lv-1) - E(s,t),
        // s = t being an empty column.
        for (int t = 1 + tid; t <= k; t += T) {
          real wv = Rl[KS + t];
          for (int l = 2; l <= lmax; ++l) {
            wv = BT::max(wv, Rl[l * KS + t]);
            Rl[l * KS + t] = wv;
          }
        }
        __syncthreads();
        for (int l = 2 + warp; l <= lmax; l += NW) {
          int tcur = k;
          for (int lv = l; lv >= 2; --lv) {
            real best = NINF;
            int arg = 0x7fffffff;
            for (int s = lv - 1 + lane; s <= tcur; s += 32) {
              const real wv = Rl[(lv - 1) * KS + s];
              const real cand = (s == tcur) ? wv : wv - Et[tri_row(s, k) + tcur - s - 1];
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
          if (lane == 0) Iw[l] = HQ + (double)Rl[l * KS + k] / (double)n;
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
        real w = Rl[KS + k];
        for (int lv = 2; lv <= lc; ++lv) w = BT::max(w, Rl[lv * KS + k]);
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

cudaError_t dp_mid_configure(bool fp32, int smem, int threads, int* blocks_per_sm, bool set_attr) {
  cudaError_t e = cudaSuccess;
  if (fp32) {
    if (set_attr)
      e = allow_dynamic_smem(reinterpret_cast<const void*>(k_dp_mid<float>), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_mid<float>, threads, smem);
  }
  if (set_attr)
    e = allow_dynamic_smem(reinterpret_cast<const void*>(k_dp_mid<double>), smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dp_mid<double>, threads, smem);
}

cudaError_t dp_mid_launch(bool fp32, int grid, int threads, int smem, cudaStream_t st,
                          const DPParams& P, const MidPlan& S) {
  if (fp32)
    k_dp_mid<float><<<grid, threads, smem, st>>>(P, S);
  else
    k_dp_mid<double><<<grid, threads, smem, st>>>(P, S);
  return cudaGetLastError();
}

}  // namespace gm
