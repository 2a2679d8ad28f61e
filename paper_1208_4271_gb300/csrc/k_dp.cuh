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
// Warp 0 solves block b (its part B) while the other warps work through the
// items of block b+1 from a shared counter: the A1 s-chunks, the entries of
// block b+1's in-block entropy triangle (once warp 0 holds block b's in
// registers), then the A2 s-chunks, which wait for warp 0 to publish block
// b's rows; warp 0 joins when it is done, and one barrier per block ends the
// step.  In A1/A2 each lane computes E(s,t) once and updates the running
// maxima of a group of levels with R(s,l-1) - E (the R row is a warp-wide
// 16-byte broadcast); the warps' partial maxima meet in shared memory
// through atomicMin on the value bits (every value is -0.0, negative or
// -inf, so a larger value has smaller bits).  Levels beyond a task's last
// level hold -inf, so no candidate needs a guard.
#pragma once
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
// Every value the DP compares -- R, W, their candidates R - E (E >= +0) and
// the -inf of unused levels -- lies in [-inf, -0.0]: a sum of negated
// entropy terms.  On that range the order of the values is the reverse of
// the order of their bit patterns, so the maximum of doubles is the minimum
// of their 64-bit patterns.  That runs on the integer pipe; GB300's FP64 pipe
// executes two operations per clock and SM, and is left the subtractions.
template <>
struct Bits<double> {
  using U = unsigned long long;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
  __device__ static double from(U b) { return __longlong_as_double((long long)b); }
  __device__ static double ninf() { return __longlong_as_double((long long)0xfff0000000000000ull); }
  __device__ static double max(double a, double b) {
    const U x = of(a), y = of(b);
    return from(y < x ? y : x);
  }
};

// The superclump data of a task in shared memory, s-major: row s holds
// sd[s*SW] = c_s (the sorted position where superclump s ends) and
// sd[s*SW + 1 + r] = cum[r][s] for the yhat rows r, SW = yhat + 1 rounded up
// to a multiple of 4 (so that a row is whole 16-byte words).
__host__ __device__ __forceinline__ int sd_width(int yhat) { return (yhat + 1 + 3) & ~3; }

// E(s,t) = L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s]), increasing r
template <typename real, typename LT>
__device__ __forceinline__ real entropy_term(const LT* __restrict__ Lt, const int* __restrict__ sd,
                                             int SW, int yhat, int s, int t) {
  const int* __restrict__ ct = sd + t * SW;
  const int* __restrict__ cs = sd + s * SW;
  real e = (real)Lt[ct[0] - cs[0]];
  int r = 1;
  // four rows at a time: the loads run ahead, the subtractions keep the
  // order of increasing r
  for (; r + 3 <= yhat; r += 4) {
    const real l0 = Lt[ct[r + 0] - cs[r + 0]];
    const real l1 = Lt[ct[r + 1] - cs[r + 1]];
    const real l2 = Lt[ct[r + 2] - cs[r + 2]];
    const real l3 = Lt[ct[r + 3] - cs[r + 3]];
    e -= l0;
    e -= l1;
    e -= l2;
    e -= l3;
  }
  for (; r <= yhat; ++r) e -= (real)Lt[ct[r] - cs[r]];
  return e;
}

// The same E(s,t) for a fixed t whose row td (yhat <= 7) sits in registers:
// row s comes in one or two 16-byte broadcast loads.
template <typename real>
__device__ __forceinline__ real entropy_reg(const real* __restrict__ Lt, const int* __restrict__ sd,
                                            int SW, int yhat, const int (&td)[8], int s) {
  const int4 a = *reinterpret_cast<const int4*>(sd + s * SW);
  real e = Lt[td[0] - a.x];
  if (yhat > 0) e -= Lt[td[1] - a.y];
  if (yhat > 1) e -= Lt[td[2] - a.z];
  if (yhat > 2) e -= Lt[td[3] - a.w];
  if (yhat > 3) {
    const int4 b = *reinterpret_cast<const int4*>(sd + s * SW + 4);
    e -= Lt[td[4] - b.x];
    if (yhat > 4) e -= Lt[td[5] - b.y];
    if (yhat > 5) e -= Lt[td[6] - b.z];
    if (yhat > 6) e -= Lt[td[7] - b.w];
  }
  return e;
}

// E(s,t) with row t in registers for a fixed row width SWC (4 or 8): the
// columns beyond yhat are 0 in both rows, and L(0) = 0, so the extra terms
// subtract exactly zero; no branch on yhat.
template <typename real, int SWC>
__device__ __forceinline__ real entropy_regc(const real* __restrict__ Lt, const int* __restrict__ sd,
                                             const int (&td)[8], int s) {
  const int4 a = *reinterpret_cast<const int4*>(sd + s * SWC);
  real e = Lt[td[0] - a.x];
  e -= Lt[td[1] - a.y];
  e -= Lt[td[2] - a.z];
  e -= Lt[td[3] - a.w];
  if constexpr (SWC == 8) {
    const int4 b = *reinterpret_cast<const int4*>(sd + s * SWC + 4);
    e -= Lt[td[4] - b.x];
    e -= Lt[td[5] - b.y];
    e -= Lt[td[6] - b.z];
    e -= Lt[td[7] - b.w];
  }
  return e;
}

// max(a, b, c) in one instruction (three-operand max.f32 of sm_100 and later)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ double fmax3(double a, double b, double c) {
  return Bits<double>::max(Bits<double>::max(a, b), c);  // values in [-inf, -0.0]
}

// (r0 - e, r1 - e) for two floats packed in 64 bits (r0 in the low half)
// in one instruction (sub.f32x2 of sm_100 and later); each element rounds
// as the scalar subtraction does
__device__ __forceinline__ float2 sub_x2(unsigned long long r, unsigned long long ee) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(r), "l"(ee));
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(d));
  return v;
}
__device__ __forceinline__ unsigned long long splat_x2(float e) {
  unsigned long long v;
  asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(e));
  return v;
}

// Prefetch into L1 of the line holding p (a hint: no fault, no result).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// With the R table in global memory, phase A copies the rows of its s-range
// into a per-warp shared-memory buffer kStageRows at a time (coalesced
// 16-byte loads, the next rows prefetched into L1 meanwhile) and reads them
// there as broadcasts; kDPStageBytes per warp hold kStageRows rows of up to
// 160 bytes (40 float or 20 double levels per pass).
constexpr int kStageRows = kDPStageRows;

// Candidates R(s, l-1) - E(s, t) for s in [s_lo, s_hi] and the LEV levels of
// one pass, max-accumulated into acc; row s of the pass's R columns starts at
// Rb + (s - s_base) * RS.  Two s per iteration: each level takes both
// candidates in one three-operand max (in float two levels share one packed
// subtraction), and the E pair of the next iteration is formed meanwhile.
// REG: 4 or 8 = row t in registers, that many columns; 1 = row t in
// registers, yhat terms; 0 = both rows from shared memory.
template <typename real, int LEV, int REG>
__device__ __forceinline__ void accumulate_rows(real (&acc)[LEV], const real* __restrict__ Rb, int RS,
                                                int s_base, int s_lo, int s_hi,
                                                const real* __restrict__ Lt,
                                                const int* __restrict__ sd, int SW, int yhat,
                                                const int (&td)[8], int tt,
                                                const int* __restrict__ sdr, int sd_off) {
  using BT = Bits<real>;
  constexpr int VW = 16 / sizeof(real);
  // (the short rows of s at sdr + (s - sd_off) * REG: sd itself, or staged)
  auto E = [&](int s) -> real {
    if constexpr (REG == 4 || REG == 8) return entropy_regc<real, REG>(Lt, sdr, td, s - sd_off);
    else if constexpr (REG == 1) return entropy_reg<real>(Lt, sd, SW, yhat, td, s);
    else return entropy_term<real>(Lt, sd, SW, yhat, s, tt);
  };
  int s = s_lo;
  if (s < s_hi) {
    real e0 = E(s), e1 = E(s + 1);
#pragma unroll 1
    for (; s + 1 <= s_hi; s += 2) {
      const bool more = s + 3 <= s_hi;
      const real n0 = more ? E(s + 2) : e0;
      const real n1 = more ? E(s + 3) : e1;
      const real* R0 = Rb + (s - s_base) * RS;
      const real* R1 = R0 + RS;
      unsigned long long ee0 = 0, ee1 = 0;
      if constexpr (sizeof(real) == 4) {
        ee0 = splat_x2(e0);
        ee1 = splat_x2(e1);
      }
#pragma unroll
      for (int g = 0; g < LEV / VW; ++g) {
        if constexpr (sizeof(real) == 4) {
          // four levels of rows s and s+1, two subtractions per instruction
          const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(R0 + 4 * g);
          const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(R1 + 4 * g);
          const float2 a0 = sub_x2(a.x, ee0), a1 = sub_x2(a.y, ee0);
          const float2 b0 = sub_x2(b.x, ee1), b1 = sub_x2(b.y, ee1);
          acc[4 * g + 0] = fmax3(acc[4 * g + 0], a0.x, b0.x);
          acc[4 * g + 1] = fmax3(acc[4 * g + 1], a0.y, b0.y);
          acc[4 * g + 2] = fmax3(acc[4 * g + 2], a1.x, b1.x);
          acc[4 * g + 3] = fmax3(acc[4 * g + 3], a1.y, b1.y);
        } else {
          const double2 a = *reinterpret_cast<const double2*>(R0 + 2 * g);
          const double2 b = *reinterpret_cast<const double2*>(R1 + 2 * g);
          acc[2 * g + 0] = fmax3(acc[2 * g + 0], a.x - e0, b.x - e1);
          acc[2 * g + 1] = fmax3(acc[2 * g + 1], a.y - e0, b.y - e1);
        }
      }
      e0 = n0;
      e1 = n1;
    }
  }
  if (s == s_hi) {  // an odd count: the last s alone
    const real e = E(s);
    const real* Rs = Rb + (s - s_base) * RS;
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
  }
}

// The same for R rows in shared memory, row s at Rt + s * LS + (lc - 2)
// (a copy of its own: sharing accumulate_rows cost the y = 2 launch 2 %
// through a different schedule).
template <typename real, int LEV, int REG>
__device__ __forceinline__ void accumulate_smem(real (&acc)[LEV], const real* __restrict__ Rt, int LS,
                                           int lc, int s_lo, int s_hi, const real* __restrict__ Lt,
                                           const int* __restrict__ sd, int SW, int yhat,
                                           const int (&td)[8], int tt) {
  using BT = Bits<real>;
  constexpr int VW = 16 / sizeof(real);
  auto E = [&](int s) -> real {
    if constexpr (REG == 4 || REG == 8) return entropy_regc<real, REG>(Lt, sd, td, s);
    else if constexpr (REG == 1) return entropy_reg<real>(Lt, sd, SW, yhat, td, s);
    else return entropy_term<real>(Lt, sd, SW, yhat, s, tt);
  };
  int s = s_lo;
  if (s < s_hi) {
    real e0 = E(s), e1 = E(s + 1);
#pragma unroll 1
    for (; s + 1 <= s_hi; s += 2) {
      const bool more = s + 3 <= s_hi;
      const real n0 = more ? E(s + 2) : e0;
      const real n1 = more ? E(s + 3) : e1;
      const real* R0 = Rt + s * LS + (lc - 2);
      const real* R1 = R0 + LS;
      unsigned long long ee0 = 0, ee1 = 0;
      if constexpr (sizeof(real) == 4) {
        ee0 = splat_x2(e0);
        ee1 = splat_x2(e1);
      }
#pragma unroll
      for (int g = 0; g < LEV / VW; ++g) {
        if constexpr (sizeof(real) == 4) {
          // four levels of rows s and s+1, two subtractions per instruction
          const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(R0 + 4 * g);
          const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(R1 + 4 * g);
          const float2 a0 = sub_x2(a.x, ee0), a1 = sub_x2(a.y, ee0);
          const float2 b0 = sub_x2(b.x, ee1), b1 = sub_x2(b.y, ee1);
          acc[4 * g + 0] = fmax3(acc[4 * g + 0], a0.x, b0.x);
          acc[4 * g + 1] = fmax3(acc[4 * g + 1], a0.y, b0.y);
          acc[4 * g + 2] = fmax3(acc[4 * g + 2], a1.x, b1.x);
          acc[4 * g + 3] = fmax3(acc[4 * g + 3], a1.y, b1.y);
        } else {
          const double2 a = *reinterpret_cast<const double2*>(R0 + 2 * g);
          const double2 b = *reinterpret_cast<const double2*>(R1 + 2 * g);
          acc[2 * g + 0] = fmax3(acc[2 * g + 0], a.x - e0, b.x - e1);
          acc[2 * g + 1] = fmax3(acc[2 * g + 1], a.y - e0, b.y - e1);
        }
      }
      e0 = n0;
      e1 = n1;
    }
  }
  if (s == s_hi) {  // an odd count: the last s alone
    const real e = E(s);
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
  }
}

// Phase A over s in [s_lo, s_hi] for the levels from lc: straight from the
// R table in shared memory, or (GS: the R table in global memory) through
// the warp's staging buffer, kStageRows rows at a time, the next rows (and
// with sdg their superclump rows) prefetched into L1 before each copy.
template <typename real, int LEV, int REG, bool GS>
__device__ __forceinline__ void accumulate(real (&acc)[LEV], const real* __restrict__ Rt, int LS,
                                           int lc, int s_lo, int s_hi, const real* __restrict__ Lt,
                                           const int* __restrict__ sd, int SW, int yhat,
                                           const int (&td)[8], int tt, real* __restrict__ stage,
                                           int lane, bool sdg) {
  if constexpr (!GS) {
    accumulate_smem<real, LEV, REG>(acc, Rt, LS, lc, s_lo, s_hi, Lt, sd, SW, yhat, td, tt);
  } else {
    constexpr int VW = 16 / sizeof(real);
    constexpr int UPR = LEV / VW;  // 16-byte units per row
    static_assert(LEV * sizeof(real) <= 160, "a staged row holds at most 160 bytes");
    for (int sb = s_lo; sb <= s_hi; sb += kStageRows) {
      const int se = min(s_hi, sb + kStageRows - 1);
      // the next rows into L1 while this copy and its candidates run
      {
        // two lanes per row (its three lines at most: first, middle, last byte)
        const int sp = se + 1 + (lane >> 1);
        if (sp <= s_hi) {
          constexpr int RB = LEV * (int)sizeof(real);
          const char* p0 = reinterpret_cast<const char*>(Rt + sp * LS + (lc - 2));
          if (lane & 1) {
            prefetch_l1(p0 + RB - 1);
          } else {
            prefetch_l1(p0);
            prefetch_l1(p0 + RB / 2);
            if (sdg) prefetch_l1(sd + sp * SW);
          }
        }
      }
      __syncwarp();  // the previous rows are read
      const int units = (se - sb + 1) * UPR;
      for (int i = lane; i < units; i += 32) {
        const int r = i / UPR, u = i - r * UPR;
        reinterpret_cast<uint4*>(stage)[i] =
            *reinterpret_cast<const uint4*>(Rt + (sb + r) * LS + (lc - 2) + u * VW);
      }
      // short superclump rows in global memory: staged beside them
      constexpr bool SDS = REG == 4 || REG == 8;
      int* sds = reinterpret_cast<int*>(reinterpret_cast<char*>(stage) + kStageRows * 160);
      if (SDS && sdg) {
        const int su = (se - sb + 1) * (REG / 4);
        for (int i = lane; i < su; i += 32)
          reinterpret_cast<int4*>(sds)[i] = reinterpret_cast<const int4*>(sd + sb * REG)[i];
      }
      __syncwarp();
      if (SDS && sdg)
        accumulate_rows<real, LEV, REG>(acc, stage, LEV, sb, sb, se, Lt, sd, SW, yhat, td, tt, sds, sb);
      else
        accumulate_rows<real, LEV, REG>(acc, stage, LEV, sb, sb, se, Lt, sd, SW, yhat, td, tt, sd, 0);
    }
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

// Iterations of a bounded wait (under a tenth of a second with the sleep in
// each); a wait that runs out marks the task's pair GMINE_E_TIMEOUT, and the
// task's later waits return at once.  (Warp 0 publishes each block after its
// in-block step, which waits on nothing: the bound is a safety net.)
constexpr unsigned kWaitLimit = 1u << 20;

// Lane 0 waits until *ready >= want (warp 0 stores the number of blocks
// whose R rows are final after a block-scope fence), then the warp goes on.
__device__ __forceinline__ void wait_ready(const int* ready, int want, int lane, bool& late) {
  if (lane == 0 && !late) {
    const volatile int* r = ready;
    unsigned it = 0;
    while (*r < want) {
      if (++it > kWaitLimit) {
        late = true;
        break;
      }
      __nanosleep(64);
    }
    __threadfence_block();
  }
  __syncwarp();
}

// Entries of the in-block entropy triangle of the block starting at t0:
// E(t0+i, t0+j), 0 <= i < j <= 31, at j(j-1)/2 + i (those with t0+j <= k).
constexpr int kEbEntries = 32 * 31 / 2;
__device__ __forceinline__ int tri_column(int p) {  // j with j(j-1)/2 <= p < j(j+1)/2
  int j = (int)((1.0f + sqrtf(8.0f * (float)p + 1.0f)) * 0.5f);
  while (j * (j - 1) / 2 > p) --j;
  while (j * (j + 1) / 2 <= p) ++j;
  return j;
}
template <typename real>
__device__ __forceinline__ void in_block_entropies(real* __restrict__ Eb, const real* __restrict__ Lt,
                                                   const int* __restrict__ sd, int SW, int yhat, int t0,
                                                   int k, int u, int U) {
  for (int p = u; p < kEbEntries; p += U) {
    const int j = tri_column(p);
    if (t0 + j <= k) Eb[p] = entropy_term<real>(Lt, sd, SW, yhat, t0 + (p - j * (j - 1) / 2), t0 + j);
  }
}

// The work for block b+1 (t in [t1, t1 + 32)) while warp 0 solves block b,
// in items from one shared counter, LEV levels per pass:
//   A1 s-chunks of CH1, s in [1, t0) (rows final before block b);
//   block b+1's in-block triangle, 32 entries per item, into EbN (a buffer
//   of its own, or, with eb_wait, block b's once warp 0 holds that in
//   registers: *ebfree >= want);
//   A2 s-chunks of 32/NW (at least 4), s in block b [t0, t1): these wait
//   until warp 0 has published block b's rows (*ready >= want).
// The A items of a pass share the running maxima, flushed into the X rows of
// block b+1 by atomicMin on the value bits when the pass changes.
template <typename real, int LEV, bool RSM>
__device__ __forceinline__ void block_items(const real* __restrict__ Rt, int LS, int lmax, int t0,
                                            int t1, int k, int* cnt, const int* ready,
                                            const int* ebfree, int want,
                                            const real* __restrict__ Lt, const int* __restrict__ sd,
                                            int SW, int yhat, int tt, bool tv,
                                            typename Bits<real>::U* Xrow, real* __restrict__ EbN,
                                            bool eb_wait, int NW, int lane, bool& late,
                                            bool sdg, real* __restrict__ stage) {
  using BT = Bits<real>;
  constexpr bool fp32 = sizeof(real) == 4;
  constexpr int nT = (kEbEntries + 31) / 32;
  const int nlev = lmax - 1;
  const int npass = (nlev + LEV - 1) / LEV;
  // s per A1 item (measured: 64 for the float instances of 24 levels and
  // more, 32 below; 16 on the double path, whose passes split the levels)
  constexpr int CH1 = !fp32 ? 16 : LEV >= 24 ? 64 : 32;
  const int nsb1 = (t0 - 1 + CH1 - 1) / CH1;
  const int nA1 = npass * nsb1;
  const int n2 = min(NW, 8);  // A2 items per pass
  const int ch2 = 32 / n2;
  const int total = nA1 + nT + npass * n2;
  // this lane's row t in registers when it is short
  const bool reg = yhat <= 7;
  int td[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) td[c] = (reg && c < SW) ? sd[tt * SW + c] : 0;
  real acc[LEV];
  int cur_pass = -1;
  bool waited = false, waited_eb = false;
  for (;;) {
    int gg = 0;
    if (lane == 0) gg = atomicAdd(cnt, 1);
    const int g = __shfl_sync(0xffffffffu, gg, 0);
    if (g >= total) break;
    int pass, s_lo, s_hi;
    if (g < nA1) {
      pass = g / nsb1;
      s_lo = 1 + (g - pass * nsb1) * CH1;
      s_hi = min(t0 - 1, s_lo + CH1 - 1);
    } else if (g < nA1 + nT) {
      if (eb_wait && !waited_eb) {
        wait_ready(ebfree, want, lane, late);
        waited_eb = true;
      }
      const int p = (g - nA1) * 32 + lane;
      if (p < kEbEntries) {
        const int j = tri_column(p);
        if (t1 + j <= k)
          EbN[p] = entropy_term<real>(Lt, sd, SW, yhat, t1 + (p - j * (j - 1) / 2), t1 + j);
      }
      continue;
    } else {
      const int h = g - nA1 - nT;
      pass = h / n2;
      s_lo = t0 + (h - pass * n2) * ch2;
      s_hi = s_lo + ch2 - 1;
      if (!waited) {
        wait_ready(ready, want, lane, late);
        waited = true;
      }
    }
    if (pass != cur_pass) {
      if (cur_pass >= 0 && tv) flush<real, LEV>(acc, Xrow, 2 + cur_pass * LEV, lmax);
#pragma unroll
      for (int i = 0; i < LEV; ++i) acc[i] = BT::ninf();
      cur_pass = pass;
    }
    // float: the row width's fixed number of terms, no branch on yhat; double:
    // only yhat terms (the padding terms would cost FP64 issue slots)
    if (reg && fp32 && SW == 4)
      accumulate<real, LEV, 4, !RSM>(acc, Rt, LS, 2 + pass * LEV, s_lo, s_hi, Lt, sd, SW, yhat, td, tt,
                                       stage, lane, sdg);
    else if (reg && fp32)
      accumulate<real, LEV, 8, !RSM>(acc, Rt, LS, 2 + pass * LEV, s_lo, s_hi, Lt, sd, SW, yhat, td, tt,
                                       stage, lane, sdg);
    else if (reg)
      accumulate<real, LEV, 1, !RSM>(acc, Rt, LS, 2 + pass * LEV, s_lo, s_hi, Lt, sd, SW, yhat, td, tt,
                                       stage, lane, sdg);
    else
      accumulate<real, LEV, 0, !RSM>(acc, Rt, LS, 2 + pass * LEV, s_lo, s_hi, Lt, sd, SW, yhat, td, tt,
                                       stage, lane, sdg);
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
  if (nlev <= 36) return 36;
  return 40;
}

// The candidates of block b with s inside the block, level after level:
// lane j owns t0+j and keeps the column E(t0+i, t0+j), i < j, in registers
// (+inf for i >= j, so those candidates are -inf).  At level l the 32
// values R(t0+i, l-1) of the previous level sit in a 32-entry buffer and
// reach every lane as eight 16-byte broadcast loads (two buffers, one per
// level parity); R(t0+j, l) is the maximum of the partial X(t0+j, l) from
// the earlier blocks and the in-block candidates.  The chain is the levels,
// each about sixty instructions, for any number of levels.
template <typename real>
__device__ __forceinline__ void phase_b_level(real* __restrict__ Rt, real* __restrict__ Rtop, int LS,
                                              int LX, int lmax, int t0, int k,
                                              const typename Bits<real>::U* __restrict__ Xcur,
                                              bool has_x, const real* __restrict__ Eb,
                                              real* __restrict__ rbuf, int lane,
                                              int* ebfree, int eb_val, bool xg = false) {
  using BT = Bits<real>;
  constexpr int VW = 16 / sizeof(real);
  const int t = t0 + lane;
  const bool tv = t <= k;
  real pinf;
  if constexpr (sizeof(real) == 4) pinf = __int_as_float(0x7f800000);
  else pinf = __longlong_as_double(0x7ff0000000000000ll);
  real ec[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) ec[i] = (tv && i < lane) ? Eb[lane * (lane - 1) / 2 + i] : pinf;
  // the triangle is in registers: the next block's may overwrite it (with
  // a single triangle buffer)
  if (ebfree) {
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      *reinterpret_cast<volatile int*>(ebfree) = eb_val;
    }
  }
  real rcur = tv ? Rt[t * LS] : BT::ninf();  // level 1
  const typename Bits<real>::U* xr = Xcur + lane * LX;
  int par = 0;
#pragma unroll 1
  for (int l = 2; l <= lmax; ++l) {
    real* rb = rbuf + par * 32;
    // the partial maximum from the earlier blocks does not depend on the
    // chain: read it before the broadcast
    // (X rows in global memory: the lane's next 32 levels into L1)
    if (xg && ((l - 2) & 31) == 0) prefetch_l1(xr + l + 31);
    const real xl = has_x ? BT::from(xr[l - 1]) : BT::ninf();
    rb[lane] = rcur;
    __syncwarp();
    // four independent running maxima (shorter dependency chains); the
    // maximum is exact, so their order does not change the result
    real m0 = xl, m1 = BT::ninf(), m2 = BT::ninf(), m3 = BT::ninf();
#pragma unroll
    for (int q = 0; q < 32 / VW; ++q) {
      if constexpr (sizeof(real) == 4) {
        const float4 r = reinterpret_cast<const float4*>(rb)[q];
        if (q & 1) {
          m2 = fmax3(m2, r.x - ec[4 * q + 0], r.y - ec[4 * q + 1]);
          m3 = fmax3(m3, r.z - ec[4 * q + 2], r.w - ec[4 * q + 3]);
        } else {
          m0 = fmax3(m0, r.x - ec[4 * q + 0], r.y - ec[4 * q + 1]);
          m1 = fmax3(m1, r.z - ec[4 * q + 2], r.w - ec[4 * q + 3]);
        }
      } else {
        const double2 r = reinterpret_cast<const double2*>(rb)[q];
        if (q & 1) {
          m2 = BT::max(m2, r.x - ec[2 * q + 0]);
          m3 = BT::max(m3, r.y - ec[2 * q + 1]);
        } else {
          m0 = BT::max(m0, r.x - ec[2 * q + 0]);
          m1 = BT::max(m1, r.y - ec[2 * q + 1]);
        }
      }
    }
    const real v = BT::max(fmax3(m0, m1, m2), m3);
    if (tv) {
      if (l != lmax) Rt[t * LS + (l - 1)] = v;
      else if (t == k) *Rtop = v;  // the last level is read at t = k only
    }
    rcur = tv ? v : BT::ninf();
    par ^= 1;
  }
}

// Launch bounds: FP32 instances with at most 20 levels per pass run as
// 128-thread CTAs, five per SM (at most 102 registers: their shared-memory
// plans are small, so more tasks in flight pay more than registers); the
// others as 128- or 256-thread CTAs, two 256-thread ones per SM.
template <typename real, bool RSM, int LEV>
__global__ void __launch_bounds__(sizeof(real) == 4 && LEV <= 20 ? 128 : 256,
                                  sizeof(real) == 4 ? (LEV <= 20 ? 5 : 2) : 1)
k_dp(DPParams P, DPPlan S) {
  using BT = Bits<real>;
  using U = typename BT::U;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_task;
  __shared__ int s_cnt[2];  // work counters of the block steps, by parity
  __shared__ int s_ready;   // blocks whose R rows are final
  __shared__ int s_ebfree;  // blocks whose triangle warp 0 holds in registers
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int NW = T >> 5;
  constexpr bool fp32 = sizeof(real) == 4;

  // R table [kmax+1][LS]: R(t, l) at column l-1 for the source levels
  // l = 1..lmax-1 (row s = 0 at -inf); the last level lmax only at t = k, in
  // *Rtop (nothing reads it elsewhere: it is no level's source).
  // Shared memory (RSM) or, for very large B, global memory.
  real* Rt = RSM ? reinterpret_cast<real*>(sm + S.off_R)
                 : reinterpret_cast<real*>(P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta);
  real* Rtop = reinterpret_cast<real*>(sm + S.off_Rtop);  // R(k, lmax)
  // [2][32][LX] bits: shared memory, or (many levels in double) the CTA's
  // global scratch
  // (with the R table in shared memory they always are: RSM keeps the
  // pointer a shared-memory one at compile time)
  U* Xb = (RSM || S.off_X >= 0) ? reinterpret_cast<U*>(sm + S.off_X)
                                : reinterpret_cast<U*>(P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta + S.x_scr_off);
  // E(t0+i, t0+j) at j(j-1)/2 + i, i < j: with two buffers block b's in
  // buffer b % 2; with one, block b's until warp 0 has taken it into
  // registers, then block b+1's
  real* Eb = reinterpret_cast<real*>(sm + S.off_Eb);
  real* Eb2 = S.off_Eb2 >= 0 ? reinterpret_cast<real*>(sm + S.off_Eb2) : Eb;
  // this warp's staging buffer of R rows (R table in global memory)
  real* stage = RSM ? nullptr : reinterpret_cast<real*>(sm + S.off_stage + warp * kDPStageBytes);
  real* rbuf = reinterpret_cast<real*>(sm + S.off_rbuf);  // [2][32]
  // [kmax+1][SW]: shared memory, or (global R table, very large k) after
  // the R table in the CTA's scratch
  int* sd = (!RSM && S.off_sd < 0)
                ? reinterpret_cast<int*>(P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta + S.sd_scr_off)
                : reinterpret_cast<int*>(sm + S.off_sd);
  // after the DP the traceback scratch (aliased on the X buffers when they
  // are in shared memory)
  int* cuts = (!RSM && S.cuts_scr_off >= 0)                               // [8 NW or NW][xmax]
                  ? reinterpret_cast<int*>(P.scratch + (int64_t)blockIdx.x * P.scratch_per_cta + S.cuts_scr_off)
                  : reinterpret_cast<int*>(sm + S.off_tb);
  double* Iw = reinterpret_cast<double*>(sm + S.off_tb + S.off_I_rel);    // [xmax+1]
  const int LS = S.LS;
  const int LX = S.LX;
  const real* Lt;  // L(m) = m ln m, m = 0..n
  {
    const real* Lsrc;
    if constexpr (fp32) Lsrc = P.L32; else Lsrc = P.L64;
    // in shared memory with the R table (known at compile time, so the
    // lookups are shared-memory loads); beside a global R table, in shared
    // memory when the plan has room for it
    if (RSM || S.off_L >= 0) {
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
    const int SW = sd_width(yhat);
    // record (ends, then cum row-major) -> s-major rows; unused columns 0
    for (int i = tid; i < SW * ks; i += T) {
      const int c = i / ks, j = i - c * ks;
      sd[j * SW + c] = c <= yhat ? rec[6 + c * ks + j] : 0;
    }
    if (P.trace.d_sc_ends && ks <= P.trace.sc_stride)
      for (int j = tid; j <= k; j += T) P.trace.d_sc_ends[trace_task * P.trace.sc_stride + j] = rec[6 + j];
    __syncthreads();
    // R(t, l) for 1 <= l <= lmax
    auto Rget = [&](int t, int l) -> real { return l == lmax ? *Rtop : Rt[t * LS + (l - 1)]; };  // l = lmax: t = k

    if (k >= 2) {
      for (int i = tid; i < ks * LS; i += T) Rt[i] = NINF;
      if (tid == 0) *Rtop = NINF;
      for (int i = tid; i < 2 * 32 * LX; i += T) Xb[i] = NINF_BITS;
      __syncthreads();
      for (int t = 1 + tid; t <= k; t += T) {
        const real r1 = -entropy_term<real>(Lt, sd, SW, yhat, 0, t);
        if (lmax > 1) Rt[t * LS] = r1;
        else if (t == k) *Rtop = r1;
      }
      in_block_entropies<real>(Eb, Lt, sd, SW, yhat, 1, k, tid, T);  // block 0
      if (tid == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
        s_ready = 0;
        s_ebfree = 0;
      }
      __syncthreads();

      bool late = false;
      const int nb = (k + 31) / 32;
      for (int b = 0; b < nb; ++b) {
        const int t0 = 1 + 32 * b;
        const int t1 = t0 + 32;  // first t of block b+1
        const bool next = t1 <= k;
        U* Xcur = Xb + (b & 1) * 32 * LX;
        U* Xnxt = Xb + ((b + 1) & 1) * 32 * LX;
        if (warp == 0) {
          // ---- block b, s inside the block
          phase_b_level<real>(Rt, Rtop, LS, LX, lmax, t0, k, Xcur, b > 0, (b & 1) ? Eb2 : Eb, rbuf,
                              lane, Eb2 == Eb ? &s_ebfree : nullptr, b + 1, !RSM && S.off_X < 0 && b > 0);
          // block b's X rows are consumed: cleared for block b+2; the other
          // counter is free until the next step
          for (int i = lane; i < 32 * LX; i += 32) Xcur[i] = NINF_BITS;
          if (lane == 0) s_cnt[(b + 1) & 1] = 0;
          __syncwarp();
          if (lane == 0) {
            __threadfence_block();
            *reinterpret_cast<volatile int*>(&s_ready) = b + 1;
          }
          __syncwarp();
        }
        // ---- block b+1: A1, its triangle, A2 (warp 0 joins when done)
        if (next) {
          const int tn = t1 + lane;  // this lane's t in block b+1
          const bool tnv = tn <= k;
          block_items<real, LEV, RSM>(Rt, LS, lmax, t0, t1, k, &s_cnt[b & 1], &s_ready, &s_ebfree, b + 1,
                                 Lt, sd, SW, yhat, tnv ? tn : k, tnv, Xnxt + lane * LX,
                                 ((b + 1) & 1) ? Eb2 : Eb, Eb2 == Eb, NW, lane, late,
                                 !RSM && S.off_sd < 0, stage);
        }
        __syncthreads();
      }
      if (late) atomicOr(&P.pp.flags[pl], 1 << GMINE_E_TIMEOUT);
    }

    // ---- I(l) for l = 2..x
    const bool need_paths = fp32 || P.trace.d_cuts != nullptr;
    if (k >= 2 && need_paths) {
      int* mycut = cuts + warp * S.xmax;
      if constexpr (fp32) {
        // Traceback in the R recursion.  l*(l) = the level of the largest
        // R(k, l'), l' <= l (the first in increasing l'), from one warp scan;
        // then from (k, l*) at (t, lv) an s with R(s, lv-1) - E(s, t) equal
        // to R(t, lv) (an exact match exists: a maximum is one of its
        // candidates), scanning down from t - 1 (since E >= 0, an s with
        // R(s, lv-1) below the target cannot match).  Each warp follows
        // several paths at once, one per group of G lanes, largest l first,
        // G as large as lets every path start in the first round; every path
        // is then re-scored in double.
        int* lst = reinterpret_cast<int*>(sm + S.off_tb + S.off_lst_rel);
        if (warp == 0) {
          real cbest = Rget(k, 1);
          int carg = 1;
          for (int l0 = 2; l0 <= lmax; l0 += 32) {
            const int l = l0 + lane;
            real v = l <= lmax ? Rget(k, l) : NINF;
            int a = l;
            // inclusive scan over levels: a later level wins only when larger
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
              const real ov = __shfl_up_sync(0xffffffffu, v, d);
              const int oa = __shfl_up_sync(0xffffffffu, a, d);
              if (lane >= d && !(v > ov)) {
                v = ov;
                a = oa;
              }
            }
            if (!(v > cbest)) {  // the levels before l0
              v = cbest;
              a = carg;
            }
            if (l <= lmax) lst[l] = a;
            cbest = __shfl_sync(0xffffffffu, v, 31);
            carg = __shfl_sync(0xffffffffu, a, 31);
          }
        }
        __syncthreads();
        // paths per round: G lanes per path, the largest G that still gives
        // every path a group in one round (at least 4 lanes per group)
        const int npaths = lmax - 1;  // levels 2..lmax
        int G = 32;
        while (G > 4 && (32 / G) * NW < npaths) --G;
        const int NG = 32 / G;  // groups per warp; lanes from NG * G on idle
        const int grp = lane / G, sub = lane - grp * G;
        const unsigned gmask = G == 32 ? 0xffffffffu : (1u << G) - 1u;
        int* gcut = cuts + (warp * 8 + min(grp, 7)) * S.xmax;
        for (int base = warp * NG; base < npaths; base += NW * NG) {
          const int pidx = base + grp;
          const bool act = grp < NG && pidx < npaths;  // the same in the whole group
          const int l = lmax - pidx;
          const int lstar = act ? lst[l] : 1;
          int lv = lstar, tcur = k, s0 = k - 1;
          bool going = act && lv >= 2;
          real target = going ? Rget(k, lv) : NINF;
          // row tcur in registers while it is the target's t (short rows)
          const bool reg = yhat <= 7;
          int td[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) td[c] = (reg && c < SW) ? sd[tcur * SW + c] : 0;
          while (__any_sync(0xffffffffu, going)) {
            const int s = s0 - sub;
            bool hit = false;
            if (going && s >= lv - 1) {
              // the filter value and E(s, tcur) side by side
              const real r = Rt[s * LS + (lv - 2)];
              const real e = reg ? entropy_reg<real>(Lt, sd, SW, yhat, td, s)
                                 : entropy_term<real>(Lt, sd, SW, yhat, s, tcur);
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
                  for (int c = 0; c < 8; ++c) td[c] = (reg && c < SW) ? sd[tcur * SW + c] : 0;
                } else {
                  going = false;
                }
              } else {
                s0 -= G;
              }
            }
          }
          __syncwarp();
          // -E(0,s_1) - E(s_1,s_2) - ... - E(s_{l*-1},k) in double: the
          // terms (column c, row r) spread over the group's lanes, all loads
          // independent, summed by the group's first lane
          double part = 0.0;
          if (act) {
            const int nt = lstar * (yhat + 1);
            for (int i = sub; i < nt; i += G) {
              const int c = i / (yhat + 1), r = i - c * (yhat + 1);
              const int a = c == 0 ? 0 : gcut[c - 1];
              const int bnd = c == lstar - 1 ? k : gcut[c];
              // r = 0: -L(c_b - c_a); r >= 1: + L(cum[r-1][b] - cum[r-1][a])
              const double L = P.L64[sd[bnd * SW + r] - sd[a * SW + r]];
              part += r == 0 ? -L : L;
            }
          }
          double tot = part;
          for (int j = 1; j < G; ++j) {
            const double o = __shfl_sync(0xffffffffu, part, min(lane + j, 31));
            if (sub + j < G) tot += o;
          }
          if (act && sub == 0) Iw[l] = HQ + tot / (double)n;
          if (act && P.trace.d_cuts) {
            // as l - 1 column ends: the l* - 1 cuts, then empty columns at k
            int32_t* dst = P.trace.d_cuts + trace_task * P.trace.cut_stride + (l - 2) * (l - 1) / 2;
            for (int c = sub; c < l - 1; c += G) dst[c] = c < lstar - 1 ? gcut[c] : k;
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
          if (s == k) *Rtop = BT::max(wv, *Rtop);
        }
        __syncthreads();
        for (int l = 2 + warp; l <= lmax; l += NW) {
          int tcur = k;
          for (int lv = l; lv >= 2; --lv) {
            real best = NINF;
            int arg = 0x7fffffff;
            for (int s = lv - 1 + lane; s <= tcur; s += 32) {
              const real wv = Rt[s * LS + (lv - 2)];
              const real cand = (s == tcur) ? wv : wv - entropy_term<real>(Lt, sd, SW, yhat, s, tcur);
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
        allow_dynamic_smem(reinterpret_cast<const void*>(k), smem);     \
    if (e != cudaSuccess) return e;                                                      \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem); \
  }                                                                                      \
  cudaError_t NAME##_launch(int lev, int grid, int threads, int smem, cudaStream_t st,    \
                            const DPParams& P, const DPPlan& S) {                        \
    NAME##_pick(lev)<<<grid, threads, smem, st>>>(P, S);                                 \
    return cudaGetLastError();                                                           \
  }                                                                                      \
  cudaError_t NAME##_occupancy(int lev, int smem, int threads, int* blocks_per_sm) {     \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, NAME##_pick(lev), threads, smem); \
  }                                                                                      \
  int NAME##_max_threads(int lev) {                                                      \
    cudaFuncAttributes a;                                                                \
    return cudaFuncGetAttributes(&a, NAME##_pick(lev)) == cudaSuccess ? a.maxThreadsPerBlock : 0; \
  }

}  // namespace gm
