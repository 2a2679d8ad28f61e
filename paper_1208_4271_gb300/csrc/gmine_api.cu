// gmine_api.cu -- host side of the libgmine C ABI (include/gmine.h):
// parameter checks, workspace planning, and the launch sequence of a batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "gmine.h"
#include "gmine_internal.cuh"
#include "kernels.h"

using namespace gm;

namespace {

constexpr int64_t kChunkPairs = 65536;  // largest chunk of pairs per pass
constexpr int kRankThreads = 1024;

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

#define GM_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) {                                   \
      last_cuda_error() = e_;                                  \
      return GMINE_E_CUDA;                                     \
    }                                                          \
  } while (0)

cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

int host_B(int64_t n, double alpha) { return (int)std::floor(std::pow((double)n, alpha)); }

int host_khat(int B, int y, double c) {
  const int x = B / y;
  const int k = (int)std::floor(c * (double)x);
  return k < 1 ? 1 : k;
}

int64_t host_cells(int B) {
  int64_t cells = 0;
  for (int y = 2; y <= B / 2; ++y) cells += B / y - 1;
  return cells;
}

struct DeviceInfo {
  int sms = 0;
  int smem_optin = 0;
};

int device_info(DeviceInfo* d) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GMINE_E_NODEVICE;
  if (cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GMINE_E_NODEVICE;
  if (cudaDeviceGetAttribute(&d->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return GMINE_E_NODEVICE;
  return GMINE_OK;
}

int rank_smem(int64_t n);

// Shape bounds of the tasks with row counts y in [ylo, yhi] of a batch with
// n samples and parameters (B, c).
struct TaskBounds {
  int B, R, xmax, kmax, cum_max, lmax;
  int sd_max;   // ints of the s-major superclump rows: max (k+1) * SW(y), yhat <= y
  int rec_max;  // ints of the largest task record
};

TaskBounds task_bounds(int n, int B, double c, int ylo, int yhi) {
  TaskBounds tb{};
  tb.B = B;
  tb.R = std::max(B / 2 - 1, 0);
  for (int y = std::max(ylo, 2); y <= std::min(yhi, B / 2); ++y) {
    const int kk = std::min(host_khat(B, y, c), n);
    const int x = B / y;
    tb.xmax = std::max(tb.xmax, x);
    tb.kmax = std::max(tb.kmax, kk);
    tb.cum_max = std::max(tb.cum_max, y * (kk + 1));
    tb.lmax = std::max(tb.lmax, std::min(x, kk));
    tb.sd_max = std::max(tb.sd_max, (kk + 1) * ((y + 1 + 3) & ~3));
    tb.rec_max = std::max(tb.rec_max, (6 + (kk + 1) * (y + 1) + 3) & ~3);
  }
  return tb;
}

// Shared-memory plan of the DP kernel for the tasks bounded by tb.
// *r_in_smem / *l_in_smem tell where the R table and the entropy table live.
DPPlan make_dp_plan(int n, const TaskBounds& tb, bool fp32, int threads, int smem_optin,
                    bool* r_in_smem) {
  const int rs = fp32 ? 4 : 8;
  const int NW = threads / 32;
  DPPlan S{};
  S.off_Eb2 = -1;
  S.LS = std::max(4, (tb.lmax - 1 + 3) & ~3);
  S.LX = std::max(4, (tb.lmax + 3) & ~3) | 1;
  S.xmax = std::max(tb.xmax, 2);
  const int64_t rbytes = (int64_t)(tb.kmax + 1) * S.LS * rs;
  const int64_t lbytes = (int64_t)(n + 1) * rs;
  // traceback scratch aliased on the X buffers once the DP is done (cuts of
  // up to eight paths per warp on the float path, one on the double path;
  // I(l); l*(l))
  const int64_t cuts_b = (4LL * (fp32 ? 8 : 1) * NW * S.xmax + 15) & ~int64_t(15);
  const int64_t I_b = (8LL * (S.xmax + 1) + 15) & ~int64_t(15);
  const int64_t lst_b = 4LL * (S.xmax + 1);
  const int64_t tb_bytes = cuts_b + I_b + lst_b;
  const int64_t xrows = (int64_t)2 * 32 * S.LX * rs;
  const int64_t sdbytes = 4LL * std::max(tb.sd_max, 4);
  const int reserve = 1024;
  // Shared memory: the X rows (or the traceback scratch aliased on them),
  // the in-block triangle, two R buffers of 32, R(k, lmax), the superclump
  // rows; with room for it, also the L table and the R table.
  // (with the X rows in global memory, the traceback's path buffers go
  // there too: hundreds of levels make them as large as the X rows)
  auto place = [&](bool x_smem, bool sd_smem) -> int64_t {
    int64_t fixed = 0;
    auto add = [&](int64_t b) { const int64_t at = fixed; fixed = (fixed + b + 15) & ~int64_t(15); return (int)at; };
    S.off_X = x_smem ? add(std::max<int64_t>(xrows, tb_bytes)) : -1;
    S.off_I_rel = x_smem ? (int)cuts_b : 0;
    S.off_lst_rel = x_smem ? (int)(cuts_b + I_b) : (int)I_b;
    S.off_tb = x_smem ? S.off_X : add(I_b + lst_b);
    S.off_Eb = add((int64_t)(32 * 31 / 2) * rs);  // the in-block triangle
    S.off_rbuf = add((int64_t)2 * 32 * rs);
    S.off_Rtop = add((int64_t)rs);  // R(k, lmax)
    S.off_sd = sd_smem ? add(sdbytes) : -1;
    return fixed;
  };
  int64_t fixed = place(true, true);
  const bool in_smem = fixed + rbytes + lbytes + 32 + reserve <= smem_optin;
  *r_in_smem = in_smem;
  // The CTA's global scratch: the R table (one spare row), then what does
  // not fit in shared memory.  The X rows go first (each is touched once
  // per level and block), the superclump rows only if they still do not fit
  // (they are read for every entropy term).
  int64_t scr = align256((int64_t)(tb.kmax + 2) * S.LS * rs);
  S.x_scr_off = -1;
  S.sd_scr_off = -1;
  S.cuts_scr_off = -1;
  // (a global R table comes with phase A's staging buffers of R rows, one
  // per warp, in shared memory)
  const int64_t stage_b = (int64_t)NW * kDPStageBytes;
  if (!in_smem && fixed + stage_b + reserve > smem_optin) {
    fixed = place(false, true);
    S.x_scr_off = scr;
    scr = align256(scr + xrows);
    S.cuts_scr_off = scr;
    scr = align256(scr + cuts_b);
    // the superclump rows go out too when they do not fit, or when on the
    // float path that frees room for the L table beside two CTAs per SM
    // (each entropy term reads a row and yhat + 1 table entries: one of the two
    // stays in shared memory)
    bool sd_out = fixed + stage_b + reserve > smem_optin;
    if (!sd_out && fp32 && 2 * (fixed + stage_b + reserve) > smem_optin + 1024) {
      const int64_t without = place(false, false);
      sd_out = 2 * (((without + 15) & ~int64_t(15)) + stage_b + lbytes + reserve) <= smem_optin + 1024;
      place(false, true);
    }
    if (sd_out) {
      fixed = place(false, false);
      S.sd_scr_off = scr;
      scr = align256(scr + sdbytes);
    }
  }
  S.scr_bytes = in_smem ? 0 : scr;
  int64_t o = fixed;
  S.off_stage = -1;
  if (!in_smem) {
    S.off_stage = (int)((o + 15) & ~int64_t(15));
    o = (S.off_stage + stage_b + 15) & ~int64_t(15);
  }
  if (in_smem) {
    S.off_L = (int)o;
    o = (o + lbytes + 15) & ~int64_t(15);
    S.off_R = (int)o;
    o = (o + rbytes + 15) & ~int64_t(15);
  } else {
    // the R table is in global memory; the L table still goes to shared
    // memory when that keeps two CTAs per SM (one for double values)
    const int64_t with_L = ((o + 15) & ~int64_t(15)) + lbytes;
    const int ctas = fp32 ? 2 : 1;
    if (ctas * (with_L + reserve) <= smem_optin + 1024) {
      S.off_L = (int)((o + 15) & ~int64_t(15));
      o = (with_L + 15) & ~int64_t(15);
    } else {
      S.off_L = -1;
    }
    S.off_R = -1;
  }
  S.total = (int)o;
  return S;
}

// Shared-memory layout of the partition kernel for n samples: the CTA's
// pi / tie-group maps, then one region per warp.
struct PartPlan {
  int warps, warp_smem, off_pi, off_gU, off_warps, total;
  int off_Qs, off_q, off_cgrp, off_cstart, off_scb, off_mixed, off_eb;
};

PartPlan make_part_plan(int n, const TaskBounds& tb, int warps) {
  PartPlan pp{};
  pp.warps = warps;
  const int64_t es = n > kMaxN16 ? 4 : 2;  // bytes per position (and count)
  int o = 0;
  auto add = [&](int64_t b) { const int at = o; o = (int)((o + b + 15) & ~int64_t(15)); return at; };
  pp.off_pi = add(es * n);
  pp.off_gU = add(es * n);
  pp.off_warps = o;
  o = 0;
  pp.off_Qs = add(std::max<int64_t>(es * n, es * std::max(tb.cum_max, 1) + 4));  // Qs, then counts
  pp.off_q = add(es * n);
  pp.off_cgrp = add(es * n);
  pp.off_cstart = add(es * (n + 1));
  pp.off_scb = add(es * (tb.kmax + 1));
  pp.off_mixed = add(4LL * ((n + 31) / 32 + 1));
  pp.off_eb = add(4LL * (tb.B / 2 + 2));
  pp.warp_smem = o;
  pp.total = pp.off_warps + warps * pp.warp_smem;
  return pp;
}

// Shared-memory layout of the warp-per-task DP kernel.
SmallPlan make_small_plan(int n, const TaskBounds& tb, bool fp32, int warps) {
  const int rs = fp32 ? 4 : 8;
  SmallPlan S{};
  S.LW = tb.xmax + 1;
  int o = 0;
  auto add = [&](int64_t b) { const int at = o; o = (int)((o + b + 15) & ~int64_t(15)); return at; };
  S.off_L = add((int64_t)(n + 1) * rs);
  S.off_warps = o;
  o = 0;
  S.off_E = add((int64_t)tb.kmax * (tb.kmax + 1) / 2 * rs);
  S.off_W = add((int64_t)(tb.kmax + 1) * S.LW * rs);
  S.off_A = add((int64_t)(tb.kmax + 1) * S.LW * 2);
  S.off_rec = add(4LL * std::max(tb.rec_max, 4));
  S.off_I = add(8LL * S.LW);
  S.off_cuts = add(4LL * S.LW * S.LW);
  S.warp_smem = o;
  S.total = S.off_warps + warps * S.warp_smem;
  return S;
}

// Shared-memory layout of the warp-per-task blocked DP kernel (float path)
// for the tasks bounded by tb, lev levels per row of the R table.
WarpPlan make_warp_plan(int n, const TaskBounds& tb, int lev, int warps) {
  WarpPlan S{};
  S.LS = lev;
  S.xmax = std::max(tb.xmax, 2);
  int64_t o = 0;
  auto add = [&](int64_t b) { const int64_t at = o; o = (o + b + 15) & ~int64_t(15); return (int)at; };
  S.off_L = add((int64_t)(n + 1) * 4);
  S.off_warps = (int)o;
  o = 0;
  S.off_R = add((int64_t)(tb.kmax + 1) * S.LS * 4);
  S.off_sd = add(4LL * tb.sd_max);
  S.off_rbuf = add(4LL * 64);
  S.off_Rtop = add(16);
  S.off_lst = add(4LL * (S.xmax + 1));
  S.off_I = add(8LL * (S.xmax + 1));
  S.off_cuts = add(4LL * 8 * S.xmax);
  S.warp_smem = (int)o;
  S.total = (int)std::min<int64_t>(S.off_warps + (int64_t)warps * o, 1LL << 30);
  return S;
}

// Shared-memory layout of the level-major DP kernel for the tasks bounded by tb.
MidPlan make_mid_plan(int n, const TaskBounds& tb, bool fp32, int threads) {
  const int rs = fp32 ? 4 : 8;
  const int NW = threads / 32;
  MidPlan S{};
  S.KS = (tb.kmax + 1 + 3) & ~3;
  S.xmax = std::max(tb.xmax, 2);
  int64_t o = 0;
  auto add = [&](int64_t b) { const int64_t at = o; o = (o + b + 15) & ~int64_t(15); return (int)at; };
  S.off_E = add((int64_t)tb.kmax * (tb.kmax + 1) / 2 * rs);
  S.off_R = add((int64_t)(tb.lmax + 1) * S.KS * rs);
  S.off_L = add((int64_t)(n + 1) * rs);
  S.off_rec = add(4LL * std::max(tb.rec_max, 4));
  S.off_I = add(8LL * (S.xmax + 1));
  S.off_cuts = add(4LL * NW * S.xmax);
  S.off_ecol = add(8LL * NW * (S.xmax + 1));
  S.total = (int)std::min<int64_t>(o, 1LL << 30);
  return S;
}

constexpr int kDPThreadsBig = 256;
constexpr int kDPThreadsSmall = 128;
constexpr int64_t kRecBudget = 12LL << 30;  // record bytes per chunk
constexpr int kMaxDPGroups = 16;

// One launch of the DP kernel: the tasks with row counts y in [ylo, yhi],
// whose column counts share one level group (levels kept in registers).
struct DPGroup {
  int ylo, yhi, lev, threads, ctas;
  bool rsm;
  bool small;      // warp-per-task kernel
  bool mid;        // level-major kernel
  bool two;        // two-column kernel (x = 2)
  bool warp;       // warp-per-task blocked kernel (float path)
  int tdw;         // its register row width
  int smem_two, off_two_rec, two_rec_bytes;
  WarpPlan WS;
  DPPlan S;
  SmallPlan SS;
  MidPlan MS;
  int64_t scratch_per_cta, o_scratch;
};

// Kernel plan of a chunk of pairs that have at most n used samples each
// and B <= Bc: DP launch groups, partition and sort placement, record sizes.
struct ChunkPlan {
  int64_t n;
  int B;
  TaskBounds tb;        // all row counts
  int ngroups;
  DPGroup grp[kMaxDPGroups];
  PartPlan part;
  int part_ctas;
  bool part_global;      // partition regions in global memory (large n)
  bool part_wide;        // 32-bit positions in the partition (n > 65535)
  int rank_ctas, rank_smem_bytes;  // rank_ctas > 0: sort keys in global scratch
  int64_t rank_scr_per_cta;
  int64_t rec_per_orient;  // ints of the task records of one (pair, orientation)
  int64_t cells;           // cells of M for B
  int R, bstride;          // equipartitions per slot: y = 2 .. R + 1, bounds stride
};

// Workspace layout of a batch (byte offsets from the workspace base).
struct Layout {
  int64_t n, p, n_pairs, chunk, slots;
  ChunkPlan cp;          // every chunk's plan (regular batches); the largest (uneven)
  int64_t o_partscr;     // partition regions in global memory, or -1
  int64_t partscr_bytes;
  int64_t o_rankscr;     // sort keys in global memory, or -1
  int64_t rankscr_bytes;
  int64_t o_Btab, o_L64, o_L32, o_lnt, o_recoff, o_nf;
  int64_t o_perm, o_pos, o_grp, o_gstart, o_ngroups, o_nslot;
  int64_t o_bounds, o_yhat;
  int64_t o_slot, o_nused, o_Bp, o_flags, o_dirty, o_ndirty;
  int64_t o_rec, o_Mo, o_queue;
  int64_t o_hvars, o_hpairs, o_hscores, o_hM;
  // uneven batches: one region each for the per-slot rank arrays, the
  // equipartitions, the records and M_o, whose layout each chunk sets for
  // its own sizes; the per-pair counts copied to the host; the pair order
  bool uneven;
  int n_tables;          // B tables (one per alpha, then the largest alpha's)
  int64_t o_rank, rank_bytes, o_equi, equi_bytes, rec_bytes, Mo_bytes, o_dpscr, dpscr_bytes;
  int64_t o_count, o_order;
  int64_t total;
};

int dp_occupancy(bool fp32, bool rsm, int lev, int smem, int threads, int* blocks) {
  const cudaError_t e = dp_configure(fp32, rsm, lev, smem, threads, blocks);
  if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
  return GMINE_OK;
}

// Global scratch of one CTA of the blocked DP: the R table (with one spare
// row: a level group may read past the last row's columns), then the
// superclump rows and the X rows when they do not fit in shared memory.
int64_t dp_scratch(const DPPlan& S, bool r_smem) { return r_smem ? 0 : S.scr_bytes; }

// CUDA events around the DP launches of one call (h_dp_ms of gmine_trace).
struct DPTiming {
  std::vector<cudaEvent_t> ev;
  ~DPTiming() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaError_t pair(cudaEvent_t* a, cudaEvent_t* b) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      const cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
    }
    *a = ev[ev.size() - 2];
    *b = ev[ev.size() - 1];
    return cudaSuccess;
  }
  int launches() const { return (int)(ev.size() / 2); }
  cudaError_t total_ms(double* out) const {
    double t = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float ms = 0.f;
      const cudaError_t r = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      if (r != cudaSuccess) return r;
      t += ms;
    }
    *out = t;
    return cudaSuccess;
  }
};

// CUDA events between the stages of one call (h_stage_ms of gmine_trace):
// mark(s) closes stage s, begun at the previous mark; s < 0 only starts.
struct StageTiming {
  std::vector<cudaEvent_t> ev;
  std::vector<int> stage;
  ~StageTiming() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaError_t mark(int s, cudaStream_t st) {
    cudaEvent_t e;
    const cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    stage.push_back(s);
    return cudaEventRecord(e, st);
  }
  cudaError_t sums(double* out) const {
    for (int s = 0; s < GMINE_N_STAGES; ++s) out[s] = 0.0;
    for (size_t i = 1; i < ev.size(); ++i) {
      if (stage[i] < 0) continue;
      float ms = 0.f;
      const cudaError_t r = cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      if (r != cudaSuccess) return r;
      out[stage[i]] += ms;
    }
    return cudaSuccess;
  }
};

// Tuned DP choices (gmine_set_dp_choices): per batch shape (n, B, c,
// precision) the kernel shape and CTA size of launch groups, process-wide.
struct ChoiceSet {
  int64_t n;
  int B;
  double c;
  bool fp32;
  std::vector<gmine_dp_choice> choices;
};
std::mutex g_choice_mu;
std::vector<ChoiceSet> g_choice_sets;

std::vector<gmine_dp_choice> dp_choices_for(int64_t n, int B, double c, bool fp32) {
  std::lock_guard<std::mutex> lock(g_choice_mu);
  for (const ChoiceSet& cs : g_choice_sets)
    if (cs.n == n && cs.B == B && cs.c == c && cs.fp32 == fp32) return cs.choices;
  return {};
}

int group_kind(const DPGroup& g) {
  return g.two ? GMINE_DP_TWO : g.warp ? GMINE_DP_WARP : g.mid ? GMINE_DP_MID
                 : g.small ? GMINE_DP_SMALL : GMINE_DP_BLOCKED;
}

int group_smem(const DPGroup& g) {
  return g.two ? g.smem_two : g.warp ? g.WS.total : g.mid ? g.MS.total : g.small ? g.SS.total : g.S.total;
}

// The kernel plan of a chunk whose pairs have at most n used samples and B
// at most Bc (tasks y = 2 .. Bc/2), clump factor c.
int plan_chunk(int64_t n, int B, double c, bool fp32, const DeviceInfo& dev, ChunkPlan* cp) {
  *cp = ChunkPlan{};
  cp->n = n;
  cp->B = B;
  int rc = GMINE_OK;
  cp->tb = task_bounds((int)n, B, c, 2, B / 2);
    // DP launch groups: consecutive row counts whose x - 1 share a level group
  cp->ngroups = 0;
  for (int y = 2; y <= B / 2; ++y) {
    // x = 2 (one level above the first) has a kernel of its own; row counts
    // with few levels are grouped by x (each launch is planned for its own
    // task sizes)
    const int x = B / y;
    const int lev = x == 2 ? 2 : dp_level_group(fp32, std::max(x - 1, 1));
    if (cp->ngroups > 0 && cp->grp[cp->ngroups - 1].lev == lev &&
        (lev > 4 || B / cp->grp[cp->ngroups - 1].ylo == x)) {
      cp->grp[cp->ngroups - 1].yhi = y;
    } else {
      if (cp->ngroups == kMaxDPGroups) return GMINE_E_LIMIT;
      DPGroup& g = cp->grp[cp->ngroups++];
      g = DPGroup{};
      g.ylo = g.yhi = y;
      g.lev = lev;
    }
  }
  const std::vector<gmine_dp_choice> forced = dp_choices_for(n, B, c, fp32);
  for (int gi = 0; gi < cp->ngroups; ++gi) {
    DPGroup& g = cp->grp[gi];
    const TaskBounds tg = task_bounds((int)n, B, c, g.ylo, g.yhi);
    const gmine_dp_choice* fc = nullptr;
    for (const gmine_dp_choice& ch : forced)
      if (ch.ylo == g.ylo && ch.yhi == g.yhi) fc = &ch;
    // each kernel shape: planned with CTA size `threads` (0: the size the
    // rules prefer), applied if its shared-memory plan fits; returns
    // GMINE_OK and sets *ok, or an error
    auto try_two = [&](int threads, bool* ok) -> int {
      *ok = false;
      if (g.lev != 2) return GMINE_OK;
      // the L table, then one task record per warp
      const int off = (int)(((n + 1) * (fp32 ? 4 : 8) + 15) & ~int64_t(15));
      const int recb = (4 * std::max(tg.rec_max, 4) + 15) & ~15;
      int th = threads > 0 ? threads : 256;
      if (threads <= 0)
        while (th > 32 && off + th / 32 * recb + 1024 > dev.smem_optin) th /= 2;
      const int smem = off + th / 32 * recb;
      if (smem + 1024 > dev.smem_optin) return GMINE_OK;
      int blocks = 0;
      cudaError_t e = dp_two_configure(fp32, smem, th, &blocks);
      if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
      if (blocks < 1) return GMINE_OK;
      g.two = true;
      g.off_two_rec = off;
      g.two_rec_bytes = recb;
      g.threads = th;
      g.smem_two = smem;
      g.ctas = blocks * dev.sms;
      g.scratch_per_cta = 0;
      *ok = true;
      return GMINE_OK;
    };
    auto try_warp = [&](int threads, bool* ok) -> int {
      *ok = false;
      if (!(fp32 && g.yhi <= 15 && dp_warp_supported(g.lev, 16))) return GMINE_OK;
      const int tdw = ((g.yhi + 1 + 3) & ~3) <= 8 ? 8 : 16;
      int best = 0;
      for (int w : {7, 4, 2, 1}) {
        if (threads > 0 && 32 * w != threads) continue;
        const WarpPlan wp = make_warp_plan((int)n, tg, g.lev, w);
        if (wp.total + 1024 > dev.smem_optin) continue;
        int blocks = 0;
        const cudaError_t e = dp_warp_configure(g.lev, tdw, wp.total, 32 * w, &blocks, true);
        if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
        // the CTA size that keeps the most warps resident
        if (blocks * w > best) {
          best = blocks * w;
          g.warp = true;
          g.tdw = tdw;
          g.WS = wp;
          g.threads = 32 * w;
        }
      }
      if (g.warp) {
        g.scratch_per_cta = 0;
        *ok = true;
      }
      return GMINE_OK;
    };
    auto try_mid = [&](int threads, bool* ok) -> int {
      *ok = false;
      if (!(g.lev >= 8 && g.lev <= 12)) return GMINE_OK;
      // the entropy triangle small enough for two CTAs per SM
      const int th = threads > 0 ? threads : (tg.kmax >= 96 ? 256 : 128);
      const MidPlan mp = make_mid_plan((int)n, tg, fp32, th);
      if (2 * (mp.total + 1024) > dev.smem_optin + 1024) return GMINE_OK;
      g.mid = true;
      g.threads = th;
      g.MS = mp;
      g.scratch_per_cta = 0;
      *ok = true;
      return GMINE_OK;
    };
    auto try_small = [&](int threads, bool* ok) -> int {
      *ok = false;
      if (!(g.lev <= 4 && tg.kmax <= 256 && tg.xmax <= 9)) return GMINE_OK;
      // as many warps per CTA as fit
      for (int w = 4; w >= 1 && !g.small; w >>= 1) {
        if (threads > 0 && 32 * w != threads) continue;
        const SmallPlan sp = make_small_plan((int)n, tg, fp32, w);
        if (sp.total + 1024 <= dev.smem_optin) {
          g.small = true;
          g.threads = 32 * w;
          g.SS = sp;
        }
      }
      if (g.small) {
        g.scratch_per_cta = 0;
        *ok = true;
      }
      return GMINE_OK;
    };
    auto try_blocked = [&](int threads, bool* ok) -> int {
      *ok = false;
      // CTA size: the one that keeps more warps resident per SM (more CTAs,
      // i.e. more tasks in flight, on a tie: their sequential parts overlap)
      int best_warps = -1;
      for (int th : {kDPThreadsSmall, kDPThreadsBig}) {
        if (threads > 0 && th != threads) continue;
        bool rsm = false;
        const DPPlan S = make_dp_plan((int)n, tg, fp32, th, dev.smem_optin, &rsm);
        if (S.total > dev.smem_optin) continue;
        if (th > dp_max_threads(fp32, rsm, g.lev)) continue;  // the instance's launch bound
        int blocks = 0;
        const int r = dp_occupancy(fp32, rsm, g.lev, std::max(S.total, 1), th, &blocks);
        if (r != GMINE_OK) return r;
        if (blocks * th / 32 > best_warps) {
          best_warps = blocks * th / 32;
          g.threads = th;
          g.S = S;
          g.rsm = rsm;
          g.ctas = blocks * dev.sms;
        }
      }
      if (best_warps <= 0) return GMINE_OK;
      // a second in-block triangle when it costs no resident CTA: the next
      // block's then needs no wait for warp 0
      {
        DPPlan S2 = g.S;
        S2.off_Eb2 = (S2.total + 15) & ~15;
        S2.total = (int)((S2.off_Eb2 + (int64_t)(32 * 31 / 2) * (fp32 ? 4 : 8) + 15) & ~int64_t(15));
        if (S2.total <= dev.smem_optin) {
          int b1 = 0, b2 = 0;
          int r = dp_occupancy(fp32, g.rsm, g.lev, std::max(g.S.total, 1), g.threads, &b1);
          if (r == GMINE_OK) r = dp_occupancy(fp32, g.rsm, g.lev, S2.total, g.threads, &b2);
          if (r != GMINE_OK) return r;
          if (b2 >= b1) g.S = S2;
        }
      }
      // the launch attribute must allow the chosen plan (the loop left the
      // last candidate's size in place)
      int blocks = 0;
      const int r = dp_occupancy(fp32, g.rsm, g.lev, std::max(g.S.total, 1), g.threads, &blocks);
      if (r != GMINE_OK) return r;
      g.scratch_per_cta = dp_scratch(g.S, g.rsm);
      *ok = true;
      return GMINE_OK;
    };
    bool ok = false;
    if (fc) {
      // a tuned choice for this group, applied when it is feasible here (a
      // general kernel for x = 2 takes the smallest level group)
      const int lev0 = g.lev;
      if (fc->kind != GMINE_DP_TWO && g.lev == 2) g.lev = dp_level_group(fp32, 1);
      switch (fc->kind) {
        case GMINE_DP_TWO: rc = try_two(fc->threads, &ok); break;
        case GMINE_DP_WARP: rc = try_warp(fc->threads, &ok); break;
        case GMINE_DP_MID: rc = try_mid(fc->threads, &ok); break;
        case GMINE_DP_SMALL: rc = try_small(fc->threads, &ok); break;
        case GMINE_DP_BLOCKED: rc = try_blocked(fc->threads, &ok); break;
        default: break;
      }
      if (rc != GMINE_OK) return rc;
      if (ok) continue;
      g.lev = lev0;
    }
    // the rules: x = 2 has a kernel of its own; a moderate number of levels
    // on the float path one warp per task; 8-12 levels the level-major
    // kernel; few columns the warp-per-task level-major kernel; else blocked
    rc = try_two(0, &ok);
    if (rc != GMINE_OK) return rc;
    if (ok) continue;
    if (g.lev == 2) g.lev = dp_level_group(fp32, 1);  // the table does not fit (very large n)
    for (auto f : {0, 1, 2, 3}) {
      rc = f == 0 ? try_warp(0, &ok) : f == 1 ? try_mid(0, &ok) : f == 2 ? try_small(0, &ok)
                                                                          : try_blocked(0, &ok);
      if (rc != GMINE_OK) return rc;
      if (ok) break;
    }
    if (!ok) return GMINE_E_LIMIT;
  }
  for (int gi = 0; gi < cp->ngroups; ++gi) {
    // an instance of the blocked kernel can serve several groups (row counts
    // with four levels are split by x; a two-column group may fall back to
    // it): one attribute per instance (the largest plan of its groups), then
    // each group's occupancy at its own size
    DPGroup& g = cp->grp[gi];
    auto blocked = [](const DPGroup& h) { return !(h.two || h.warp || h.mid || h.small); };
    if (!blocked(g)) continue;
    int smax = 1;
    for (int gj = 0; gj < cp->ngroups; ++gj) {
      const DPGroup& h = cp->grp[gj];
      if (blocked(h) && h.rsm == g.rsm && h.lev == g.lev) smax = std::max(smax, h.S.total);
    }
    int blocks = 0;
    cudaError_t e = dp_configure(fp32, g.rsm, g.lev, smax, g.threads, &blocks);
    if (e == cudaSuccess) e = dp_occupancy_only(fp32, g.rsm, g.lev, std::max(g.S.total, 1), g.threads, &blocks);
    if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
    if (blocks < 1) return GMINE_E_LIMIT;
    g.ctas = blocks * dev.sms;
  }
  {
    // the warp-per-task kernel is shared by its groups: one attribute (the
    // largest plan), then each group's occupancy at its own size
    int smax = 0, mmax = 0;
    for (int gi = 0; gi < cp->ngroups; ++gi) {
      if (cp->grp[gi].small) smax = std::max(smax, cp->grp[gi].SS.total);
      if (cp->grp[gi].mid) mmax = std::max(mmax, cp->grp[gi].MS.total);
    }
    for (int gi = 0; gi < cp->ngroups; ++gi) {
      DPGroup& g = cp->grp[gi];
      if (!g.mid) continue;
      int blocks = 0;
      cudaError_t e = dp_mid_configure(fp32, mmax, g.threads, &blocks, true);
      if (e == cudaSuccess) e = dp_mid_configure(fp32, g.MS.total, g.threads, &blocks, false);
      if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
      if (blocks < 1) return GMINE_E_LIMIT;
      g.ctas = blocks * dev.sms;
    }
    for (int gi = 0; gi < cp->ngroups; ++gi) {
      // one attribute per warp-kernel instance (the largest plan of its
      // groups), then each group's occupancy at its own size
      DPGroup& g = cp->grp[gi];
      if (!g.warp) continue;
      int wmax = 0;
      for (int gj = 0; gj < cp->ngroups; ++gj)
        if (cp->grp[gj].warp && cp->grp[gj].lev == g.lev && cp->grp[gj].tdw == g.tdw)
          wmax = std::max(wmax, cp->grp[gj].WS.total);
      int blocks = 0;
      cudaError_t e = dp_warp_configure(g.lev, g.tdw, wmax, g.threads, &blocks, true);
      if (e == cudaSuccess) e = dp_warp_configure(g.lev, g.tdw, g.WS.total, g.threads, &blocks, false);
      if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
      if (blocks < 1) return GMINE_E_LIMIT;
      g.ctas = blocks * dev.sms;
    }
    for (int gi = 0; gi < cp->ngroups; ++gi) {
      DPGroup& g = cp->grp[gi];
      if (!g.small) continue;
      int blocks = 0;
      cudaError_t e = dp_small_configure(fp32, smax, g.threads, &blocks);
      if (e == cudaSuccess) e = dp_small_occupancy(fp32, g.SS.total, g.threads, &blocks);
      if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
      if (blocks < 1) return GMINE_E_LIMIT;
      g.ctas = blocks * dev.sms;
    }
  }
  cp->part = make_part_plan((int)n, cp->tb, 4);
  if (cp->part.total + 1024 > dev.smem_optin) cp->part = make_part_plan((int)n, cp->tb, 1);
  const bool part_wide = n > kMaxN16;  // 32-bit positions and counts
  const bool part_global = part_wide || cp->part.total + 1024 > dev.smem_optin;
  cp->part_global = part_global;
  if (part_global) cp->part = make_part_plan((int)n, cp->tb, 4);  // in global scratch
  cp->part_wide = part_wide;
  {
    int pb = 0;
    const int smem = part_global ? 0 : cp->part.total;
    cudaError_t e = partition_configure(part_global, part_wide, smem, 32 * cp->part.warps, &pb);
    if (e != cudaSuccess) { last_cuda_error() = e; return GMINE_E_CUDA; }
    if (pb < 1) return GMINE_E_LIMIT;
    cp->part_ctas = (part_global ? std::min(pb, 4) : pb) * dev.sms;
  }
  // the sort: in shared memory up to kMaxRankN samples, else keys and indices
  // in global scratch, two resident CTAs per SM looping over the slots
  {
    int64_t N2 = 1;
    while (N2 < n) N2 <<= 1;
    cp->rank_smem_bytes = rank_smem(n);
    cp->rank_ctas = 0;
    cp->rank_scr_per_cta = 0;
    if (cp->rank_smem_bytes > dev.smem_optin) {
      cp->rank_smem_bytes = 4 * (kRankThreads + 1) + 64;
      cp->rank_ctas = 2 * dev.sms;
      cp->rank_scr_per_cta = (N2 * 12 + 255) & ~int64_t(255);
    }
  }
  cp->rec_per_orient = std::max<int64_t>(rec_offset(B, (int)n, c, B / 2 + 1), 4);
  cp->cells = std::max<int64_t>(host_cells(B), 1);
  cp->R = std::max(cp->tb.R, 1);
  cp->bstride = cp->tb.R + 2;
  return rc;
}

int make_layout(int64_t p, int64_t n, int64_t n_pairs, const gmine_param* param, int32_t precision,
                int32_t flags, Layout* L) {
  if (!param) return GMINE_E_ARG;
  if (gmine_check_param(param) != GMINE_OK) return GMINE_E_PARAM;
  if (p < 0 || n < 0 || n_pairs < 0) return GMINE_E_ARG;
  if (precision != GMINE_PLAIN_FP64 && precision != GMINE_FP32_DP_FP64_RESCORE) return GMINE_E_ARG;
  if (n > kMaxN) return GMINE_E_LIMIT;
  DeviceInfo dev;
  int rc = device_info(&dev);
  if (rc != GMINE_OK) return rc;
  *L = Layout{};
  L->n = n;
  L->p = p;
  L->n_pairs = n_pairs;
  const int B = n > 0 ? host_B(n, param->alpha) : 0;
  const bool fp32 = precision == GMINE_FP32_DP_FP64_RESCORE;
  rc = plan_chunk(n, B, param->c, fp32, dev, &L->cp);
  if (rc != GMINE_OK) return rc;
  const int64_t rec_pair = 2 * L->cp.rec_per_orient * 4;
  L->chunk = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(n_pairs, kChunkPairs),
                                                    kRecBudget / rec_pair));
  L->slots = p + 2 * L->chunk;

  const int64_t S = L->slots;
  const int R = L->cp.R;
  const int bstride = L->cp.bstride;
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    const int64_t at = o;
    o = align256(o + std::max<int64_t>(bytes, 1));
    return at;
  };
  L->partscr_bytes = L->cp.part_global ? (int64_t)L->cp.part_ctas * ((L->cp.part.total + 255) & ~255) : 0;
  L->o_partscr = L->cp.part_global ? take(L->partscr_bytes) : -1;
  L->rankscr_bytes = L->cp.rank_ctas > 0 ? (int64_t)L->cp.rank_ctas * L->cp.rank_scr_per_cta : 0;
  L->o_rankscr = L->cp.rank_ctas > 0 ? take(L->rankscr_bytes) : -1;
  L->n_tables = 2;
  L->o_Btab = take(4 * (n + 1) * L->n_tables);
  L->o_L64 = take(8 * (n + 1));
  L->o_L32 = take(4 * (n + 1));
  L->o_lnt = take(8 * (n + 1));
  L->o_recoff = take(8 * (L->cp.B / 2 + 2));
  L->o_nf = take(4 * p);
  L->o_perm = take(4 * S * n);
  L->o_pos = take(4 * S * n);
  L->o_grp = take(4 * S * n);
  L->o_gstart = take(4 * S * (n + 1));
  L->o_ngroups = take(4 * S);
  L->o_nslot = take(4 * S);
  L->o_bounds = take(4 * S * (int64_t)R * bstride);
  L->o_yhat = take(4 * S * (int64_t)R);
  L->o_slot = take(4 * 2 * L->chunk);
  L->o_nused = take(4 * L->chunk);
  L->o_Bp = take(4 * L->chunk);
  L->o_flags = take(4 * L->chunk);
  L->o_dirty = take(4 * L->chunk);
  L->o_ndirty = take(4);
  L->o_rec = take(L->chunk * rec_pair);
  L->o_Mo = take(8 * L->chunk * 2 * L->cp.cells);
  L->o_queue = take(8 * (kMaxDPGroups + 1));
  for (int gi = 0; gi < L->cp.ngroups; ++gi)
    L->cp.grp[gi].o_scratch = take(L->cp.grp[gi].scratch_per_cta * L->cp.grp[gi].ctas);
  if (flags & GMINE_PLAN_HOST_STAGING) {
    L->o_hvars = take(8 * p * n);
    L->o_hpairs = take(4 * 2 * n_pairs);
    L->o_hscores = take((int64_t)sizeof(gmine_pair_score) * n_pairs);
    L->o_hM = take(8 * n_pairs * L->cp.cells);
  } else {
    L->o_hvars = L->o_hpairs = L->o_hscores = L->o_hM = -1;
  }
  L->total = o;
  return GMINE_OK;
}

template <typename T>
T* at(void* base, int64_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

RankData rank_data(void* ws, const Layout& L) {
  RankData rk;
  rk.perm = at<int32_t>(ws, L.o_perm);
  rk.pos = at<int32_t>(ws, L.o_pos);
  rk.grp = at<int32_t>(ws, L.o_grp);
  rk.gstart = at<int32_t>(ws, L.o_gstart);
  rk.ngroups = at<int32_t>(ws, L.o_ngroups);
  rk.nslot = at<int32_t>(ws, L.o_nslot);
  rk.stride = L.n;
  return rk;
}

EquiData equi_data(void* ws, const Layout& L) {
  EquiData eq;
  eq.bounds = at<int32_t>(ws, L.o_bounds);
  eq.yhat = at<int32_t>(ws, L.o_yhat);
  eq.R = L.cp.R;
  eq.bstride = L.cp.bstride;
  return eq;
}

PairPrep pair_prep(void* ws, const Layout& L) {
  PairPrep pp{};
  pp.slot = at<int32_t>(ws, L.o_slot);
  pp.n_used = at<int32_t>(ws, L.o_nused);
  pp.B = at<int32_t>(ws, L.o_Bp);
  pp.flags = at<int32_t>(ws, L.o_flags);
  pp.dirty = at<int32_t>(ws, L.o_dirty);
  pp.ndirty = at<int32_t>(ws, L.o_ndirty);
  pp.order = nullptr;
  pp.aidx = nullptr;
  pp.btab_stride = L.n + 1;
  pp.slot0 = L.uneven ? 0 : L.p;
  pp.all_dirty = L.uneven ? 1 : 0;
  return pp;
}

int rank_smem(int64_t n) {
  int64_t N2 = 1;
  while (N2 < n) N2 <<= 1;
  return (int)(N2 * 12 + 4 * (kRankThreads + 1) + 64);
}

// B(m) = floor(m^alpha) for m = 0..n, one table per alpha and then one for
// the largest alpha, written into the workspace.
int upload_Btab(void* ws, const Layout& L, const double* alphas, int na, cudaStream_t st) {
  // one host buffer per thread, grown to the largest size seen (no device
  // allocation); the copy from pageable memory returns once the data is
  // staged, so the buffer can be reused at once
  static thread_local std::vector<int32_t> Bt;
  const int64_t stride = L.n + 1;
  const size_t need = (size_t)(stride * (na + 1));
  if (Bt.size() < need) Bt.resize(need);
  double amax = alphas[0];
  for (int a = 1; a < na; ++a) amax = std::max(amax, alphas[a]);
  for (int a = 0; a <= na; ++a) {
    const double al = a < na ? alphas[a] : amax;
    for (int64_t m = 0; m <= L.n; ++m) Bt[(size_t)(a * stride + m)] = m > 0 ? host_B(m, al) : 0;
  }
  GM_CUDA(cudaMemcpyAsync(at<int32_t>(ws, L.o_Btab), Bt.data(), sizeof(int32_t) * need,
                          cudaMemcpyHostToDevice, st));
  return GMINE_OK;
}

// Ranks and equipartitions of the clean variables (slots 0..p-1).
int prepare_variables(const double* d_vars, void* ws, const Layout& L, double alpha, double c,
                      cudaStream_t st, int* launches) {
  int rc = upload_Btab(ws, L, &alpha, 1, st);
  if (rc != GMINE_OK) return rc;
  const int n = (int)L.n;
  k_tables<<<(std::max(n, L.cp.B) + 256) / 256, 256, 0, st>>>(
      n, at<double>(ws, L.o_L64), at<float>(ws, L.o_L32), at<double>(ws, L.o_lnt), L.cp.B, n, c,
      at<int64_t>(ws, L.o_recoff));
  GM_CUDA(cudaGetLastError());
  ++*launches;
  if (L.p > 0) {
    k_nonfinite<<<(unsigned)((L.p + 7) / 8), 256, 0, st>>>(d_vars, L.p, n, at<int32_t>(ws, L.o_nf));
    GM_CUDA(cudaGetLastError());
    ++*launches;
    const int smem = L.cp.rank_smem_bytes;
    PairPrep pp = pair_prep(ws, L);
    unsigned char* rscr = L.o_rankscr >= 0 ? at<unsigned char>(ws, L.o_rankscr) : nullptr;
    const int64_t rgrid = rscr ? std::min<int64_t>(L.p, L.cp.rank_ctas) : L.p;
    GM_CUDA(rank_launch((int)rgrid, kRankThreads, smem, st, d_vars, n, n, at<int32_t>(ws, L.o_nf),
                        nullptr, 0, pp, at<int32_t>(ws, L.o_Btab), 0, L.p, rank_data(ws, L), rscr,
                        L.cp.rank_scr_per_cta));
    ++*launches;
    if (L.cp.tb.R > 0) {
      const int64_t work = L.p * L.cp.tb.R;
      k_equi<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(
          0, L.p, L.p, at<int32_t>(ws, L.o_Btab), nullptr, rank_data(ws, L), equi_data(ws, L));
      GM_CUDA(cudaGetLastError());
      ++*launches;
    }
  }
  return GMINE_OK;
}

bool plausible_device_ptr(const void* p) { return p != nullptr; }

// Working memory of one chunk of pairs (device pointers).
struct ChunkMem {
  RankData rk;
  EquiData eq;
  PairPrep pp;
  int32_t* rec;
  double* Mo;
  int64_t* rec_off;
  unsigned long long* queue;  // [kMaxDPGroups + 1]
  unsigned char* partscr;     // partition regions in global memory, if planned
  int64_t partscr_bytes;
  unsigned char* rankscr;     // sort keys in global memory, if planned
  int64_t rankscr_bytes;
  char* dpscr;                // one region for every DP group (NULL: each group's own)
  int64_t dpscr_bytes;
};

ChunkMem regular_mem(void* ws, const Layout& L) {
  ChunkMem cm{};
  cm.rk = rank_data(ws, L);
  cm.eq = equi_data(ws, L);
  cm.pp = pair_prep(ws, L);
  cm.rec = at<int32_t>(ws, L.o_rec);
  cm.Mo = at<double>(ws, L.o_Mo);
  cm.rec_off = at<int64_t>(ws, L.o_recoff);
  cm.queue = at<unsigned long long>(ws, L.o_queue);
  cm.partscr = L.o_partscr >= 0 ? at<unsigned char>(ws, L.o_partscr) : nullptr;
  cm.partscr_bytes = L.partscr_bytes;
  cm.rankscr = L.o_rankscr >= 0 ? at<unsigned char>(ws, L.o_rankscr) : nullptr;
  cm.rankscr_bytes = L.rankscr_bytes;
  cm.dpscr = nullptr;
  cm.dpscr_bytes = 0;
  return cm;
}

// Everything one batch call shares across its chunks.
struct BatchCtx {
  const double* vars;
  int64_t p, n_row;
  const int32_t* pairs;
  int64_t n_pairs;
  double c;
  bool fp32;
  void* ws;
  const Layout* L;
  const int32_t* Btab;        // the pairs' B tables
  const int32_t* Btab_slots;  // the table of the largest alpha (slots)
  const int32_t* nf;          // non-finite samples per variable (regular batches)
  gmine_pair_score* scores;
  double* M;
  int64_t m_stride;
  const gmine_trace* trace;
  DPTiming* timing;
  StageTiming* stages;
  cudaStream_t st;
  int launches;
};

// One chunk: pairs at batch positions [pair0, pair0 + C), planned by cp:
// pair slots, their own ranks and equipartitions where needed, the
// partitions of every task, the DP launches, M and the statistics.
int run_chunk(BatchCtx& b, const ChunkPlan& cp, const ChunkMem& cm, int64_t pair0, int64_t C) {
  const Layout& L = *b.L;
  cudaStream_t st = b.st;
  PairPrep pp = cm.pp;
  auto mark = [&](int s) -> cudaError_t { return b.stages ? b.stages->mark(s, st) : cudaSuccess; };
  GM_CUDA(mark(-1));
  GM_CUDA(cudaMemsetAsync(pp.ndirty, 0, 4, st));
  k_pair_prep<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(b.pairs, pair0, C, b.p, (int)b.n_row,
                                                            b.nf, b.Btab, pp);
  GM_CUDA(cudaGetLastError());
  ++b.launches;
  {
    // pairs with their own (compacted) ranks
    unsigned char* rscr = nullptr;
    int64_t rctas = 0;
    if (cp.rank_ctas > 0) {
      rscr = cm.rankscr;
      rctas = std::min<int64_t>(cp.rank_ctas, cm.rankscr_bytes / std::max<int64_t>(cp.rank_scr_per_cta, 1));
      if (!rscr || rctas < 1) return GMINE_E_WORKSPACE;
    }
    const int64_t rgrid = rscr ? std::min<int64_t>(2 * C, rctas) : 2 * C;
    GM_CUDA(rank_launch((int)rgrid, kRankThreads, cp.rank_smem_bytes, st, b.vars, b.n_row, (int)cp.n,
                        b.nf, b.pairs, pair0, pp, b.Btab, pp.slot0, 2 * C, cm.rk, rscr,
                        cp.rank_scr_per_cta));
    ++b.launches;
  }
  GM_CUDA(mark(GMINE_STAGE_PAIRS));
  if (cp.tb.R > 0) {
    const int64_t work = 2 * C * cp.tb.R;
    k_equi<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(pp.slot0, 2 * C, pp.slot0, b.Btab_slots,
                                                           pp.ndirty, cm.rk, cm.eq);
    GM_CUDA(cudaGetLastError());
    ++b.launches;
  }
  GM_CUDA(mark(GMINE_STAGE_EQUI));
  const int64_t ntasks = 2 * (int64_t)cp.tb.R * C;
  if (ntasks > 0) {
    // partition of every task of the chunk
    PartParams Q{};
    Q.rk = cm.rk;
    Q.eq = cm.eq;
    Q.pp = pp;
    Q.L64 = at<double>(b.ws, L.o_L64);
    Q.lnt = at<double>(b.ws, L.o_lnt);
    Q.rec = cm.rec;
    Q.rec_per_orient = cp.rec_per_orient;
    Q.rec_off = cm.rec_off;
    Q.B_full = cp.B;
    Q.n_full = (int)cp.n;
    Q.c = b.c;
    Q.chunk_pairs = C;
    Q.queue = cm.queue + kMaxDPGroups;
    Q.off_pi = cp.part.off_pi;
    Q.off_gU = cp.part.off_gU;
    Q.off_warps = cp.part.off_warps;
    Q.warp_smem = cp.part.warp_smem;
    Q.off_Qs = cp.part.off_Qs;
    Q.off_q = cp.part.off_q;
    Q.off_cgrp = cp.part.off_cgrp;
    Q.off_cstart = cp.part.off_cstart;
    Q.off_scb = cp.part.off_scb;
    Q.off_mixed = cp.part.off_mixed;
    Q.off_eb = cp.part.off_eb;
    Q.gscr_per_cta = (cp.part.total + 255) & ~255;
    int pctas = cp.part_ctas;
    Q.gscr = nullptr;
    if (cp.part_global) {
      Q.gscr = cm.partscr;
      pctas = (int)std::min<int64_t>(pctas, cm.partscr_bytes / Q.gscr_per_cta);
      if (!Q.gscr || pctas < 1) return GMINE_E_WORKSPACE;
    }
    // fewer (pair, orientation) jobs than twice the resident CTAs (few
    // pairs of many samples): each job's row counts are split over several
    // CTAs, interleaved
    Q.parts = (int)std::max<int64_t>(1, std::min<int64_t>(
        std::min<int64_t>(16, std::max(cp.tb.R, 1)), (2LL * pctas + 2 * C - 1) / (2 * C)));
    GM_CUDA(cudaMemsetAsync(Q.queue, 0, 8, st));
    GM_CUDA(partition_launch(cp.part_global, cp.part_wide, pctas, 32 * cp.part.warps,
                             cp.part_global ? 0 : cp.part.total, st, Q));
    GM_CUDA(cudaGetLastError());
    ++b.launches;
    GM_CUDA(mark(GMINE_STAGE_PARTITION));
    // the dynamic program: large row counts... small row counts
    DPParams P{};
    P.pp = pp;
    P.rec = Q.rec;
    P.rec_per_orient = cp.rec_per_orient;
    P.rec_off = Q.rec_off;
    P.B_full = cp.B;
    P.n_full = (int)cp.n;
    P.c = b.c;
    P.L64 = at<double>(b.ws, L.o_L64);
    P.L32 = at<float>(b.ws, L.o_L32);
    P.lnt = at<double>(b.ws, L.o_lnt);
    P.Mo = cm.Mo;
    P.cells_max = (int)cp.cells;
    P.chunk_pairs = C;
    P.counters = b.trace ? b.trace->d_counters : nullptr;
    if (b.trace) P.trace = *b.trace;
    P.trace_pair0 = pair0;
    P.trace_npairs = b.n_pairs;
    unsigned long long* qs = cm.queue;
    GM_CUDA(cudaMemsetAsync(qs, 0, 8 * kMaxDPGroups, st));
    for (int gi = 0; gi < cp.ngroups; ++gi) {
      const DPGroup& g = cp.grp[gi];
      P.task_begin = 2 * (int64_t)(g.ylo - 2) * C;
      P.task_end = 2 * (int64_t)(g.yhi - 1) * C;
      P.queue = qs + gi;
      P.scratch_per_cta = g.scratch_per_cta;
      int ctas = g.ctas;
      if (cm.dpscr) {
        P.scratch = cm.dpscr;
        if (g.scratch_per_cta > 0) {
          ctas = (int)std::min<int64_t>(ctas, cm.dpscr_bytes / g.scratch_per_cta);
          if (ctas < 1) return GMINE_E_WORKSPACE;
        }
      } else {
        P.scratch = at<char>(b.ws, g.o_scratch);
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (b.timing) {
        GM_CUDA(b.timing->pair(&e0, &e1));
        GM_CUDA(cudaEventRecord(e0, st));
      }
      if (g.two)
        GM_CUDA(dp_two_launch(b.fp32, ctas, g.threads, g.smem_two, st, P, g.off_two_rec,
                              g.two_rec_bytes));
      else if (g.warp)
        GM_CUDA(dp_warp_launch(g.lev, g.tdw, ctas, g.threads, g.WS.total, st, P, g.WS));
      else if (g.mid)
        GM_CUDA(dp_mid_launch(b.fp32, ctas, g.threads, g.MS.total, st, P, g.MS));
      else if (g.small)
        GM_CUDA(dp_small_launch(b.fp32, ctas, g.threads, g.SS.total, st, P, g.SS));
      else
        GM_CUDA(dp_launch(b.fp32, g.rsm, g.lev, ctas, g.threads, g.S.total, st, P, g.S));
      ++b.launches;
      if (b.timing) GM_CUDA(cudaEventRecord(e1, st));
    }
    GM_CUDA(mark(GMINE_STAGE_DP));
  }
  FinalParams F{};
  F.Mo = cm.Mo;
  F.cells_max = (int)cp.cells;
  F.pp = pp;
  F.chunk_pairs = C;
  F.pair0 = pair0;
  F.scores = b.scores;
  F.M = b.M;
  F.m_stride = b.m_stride;
  F.eq_yhat = cm.eq.yhat;
  F.R = cm.eq.R;
  k_final<<<(unsigned)((C + 7) / 8), 256, 0, st>>>(F);
  GM_CUDA(cudaGetLastError());
  ++b.launches;
  GM_CUDA(mark(GMINE_STAGE_FINAL));
  return GMINE_OK;
}

// The trace epilogue of a batch call: launch count and DP kernel time.
int finish_trace(const BatchCtx& b) {
  if (b.trace && b.trace->h_kernel_launches) *b.trace->h_kernel_launches = b.launches;
  if (b.stages) {
    GM_CUDA(cudaStreamSynchronize(b.st));
    GM_CUDA(b.stages->sums(b.trace->h_stage_ms));
  }
  if (b.timing) {
    GM_CUDA(cudaStreamSynchronize(b.st));
    double ms = 0.0;
    GM_CUDA(b.timing->total_ms(&ms));
    *b.trace->h_dp_ms = ms;
    if (b.trace->h_dp_launches) *b.trace->h_dp_launches = b.timing->launches();
    if (b.trace->h_launch_ms)
      for (int i = 0; i < b.timing->launches() && i < b.trace->launch_cap; ++i)
        GM_CUDA(cudaEventElapsedTime(&b.trace->h_launch_ms[i], b.timing->ev[2 * i], b.timing->ev[2 * i + 1]));
  }
  return GMINE_OK;
}

// ---- uneven batches --------------------------------------------------------

constexpr int kMaxAlphas = 8;
constexpr int64_t kUnevenRankBudget = 2LL << 30;   // per-slot rank arrays of a chunk
constexpr int64_t kUnevenEquiBudget = 2LL << 30;   // equipartitions of a chunk
constexpr int64_t kUnevenRecBudget = 24LL << 30;   // task records of a chunk
constexpr int64_t kUnevenMoBudget = 1LL << 30;     // M of both orientations of a chunk

// Bytes a chunk of C pairs with at most n samples and B <= Bc needs in each
// region of the uneven layout (sub-arrays 256-byte aligned).
struct ChunkBytes {
  int64_t rank, equi, rec, Mo;
};

ChunkBytes chunk_bytes(int64_t C, int64_t n, int B, double c) {
  ChunkBytes cb{};
  const int64_t S = 2 * C;
  cb.rank = 3 * align256(4 * S * n) + align256(4 * S * (n + 1)) + 2 * align256(4 * S);
  const int64_t R = std::max(B / 2 - 1, 1);
  cb.equi = align256(4 * S * R * (R + 2)) + align256(4 * S * R);
  cb.rec = S * std::max<int64_t>(rec_offset(B, (int)n, c, B / 2 + 1), 4) * 4;
  cb.Mo = 8 * S * std::max<int64_t>(host_cells(B), 1);
  return cb;
}

int check_alphas(const double* alphas, int na, double c) {
  if (!alphas || na < 1) return GMINE_E_ARG;
  if (na > kMaxAlphas) return GMINE_E_LIMIT;
  for (int a = 0; a < na; ++a) {
    const gmine_param prm{alphas[a], c};
    if (gmine_check_param(&prm) != GMINE_OK) return GMINE_E_PARAM;
  }
  return GMINE_OK;
}

int make_layout_uneven(int64_t p, int64_t n, int64_t n_pairs, const double* alphas, int na,
                       double c, int32_t precision, Layout* L) {
  int rc = check_alphas(alphas, na, c);
  if (rc != GMINE_OK) return rc;
  if (p < 0 || n < 0 || n_pairs < 0) return GMINE_E_ARG;
  if (precision != GMINE_PLAIN_FP64 && precision != GMINE_FP32_DP_FP64_RESCORE) return GMINE_E_ARG;
  if (n > kMaxN) return GMINE_E_LIMIT;
  DeviceInfo dev;
  rc = device_info(&dev);
  if (rc != GMINE_OK) return rc;
  *L = Layout{};
  L->uneven = true;
  L->n = n;
  L->p = p;
  L->n_pairs = n_pairs;
  double amax = alphas[0];
  for (int a = 1; a < na; ++a) amax = std::max(amax, alphas[a]);
  const int B = n > 0 ? host_B(n, amax) : 0;
  const bool fp32 = precision == GMINE_FP32_DP_FP64_RESCORE;
  // the largest chunk plan bounds the scratch regions; the others fit them
  // with fewer CTAs at most
  rc = plan_chunk(std::max<int64_t>(n, 4), B, c, fp32, dev, &L->cp);
  if (rc != GMINE_OK) return rc;
  L->chunk = std::max<int64_t>(1, std::min<int64_t>(n_pairs, kChunkPairs));
  L->n_tables = na + 1;
  const ChunkBytes one = chunk_bytes(1, std::max<int64_t>(n, 4), B, c);
  const ChunkBytes all = chunk_bytes(std::max<int64_t>(L->chunk, 1), std::max<int64_t>(n, 4), B, c);
  auto cap = [](int64_t one_pair, int64_t all_pairs, int64_t budget) {
    return std::max(one_pair, std::min(all_pairs, budget));
  };
  L->rank_bytes = cap(one.rank, all.rank, kUnevenRankBudget);
  L->equi_bytes = cap(one.equi, all.equi, kUnevenEquiBudget);
  L->rec_bytes = cap(one.rec, all.rec, kUnevenRecBudget);
  L->Mo_bytes = cap(one.Mo, all.Mo, kUnevenMoBudget);
  int64_t dps = 0;
  for (int gi = 0; gi < L->cp.ngroups; ++gi)
    dps = std::max(dps, L->cp.grp[gi].scratch_per_cta * L->cp.grp[gi].ctas);
  L->dpscr_bytes = dps;
  int64_t o = 0;
  auto take = [&](int64_t bytes) {
    const int64_t at = o;
    o = align256(o + std::max<int64_t>(bytes, 1));
    return at;
  };
  L->partscr_bytes = L->cp.part_global ? (int64_t)L->cp.part_ctas * ((L->cp.part.total + 255) & ~255) : 0;
  L->o_partscr = L->cp.part_global ? take(L->partscr_bytes) : -1;
  L->rankscr_bytes = L->cp.rank_ctas > 0 ? (int64_t)L->cp.rank_ctas * L->cp.rank_scr_per_cta : 0;
  L->o_rankscr = L->cp.rank_ctas > 0 ? take(L->rankscr_bytes) : -1;
  L->o_Btab = take(4 * (n + 1) * L->n_tables);
  L->o_L64 = take(8 * (n + 1));
  L->o_L32 = take(4 * (n + 1));
  L->o_lnt = take(8 * (n + 1));
  L->o_recoff = take(8 * (B / 2 + 2));
  L->o_rank = take(L->rank_bytes);
  L->o_equi = take(L->equi_bytes);
  L->o_slot = take(4 * 2 * L->chunk);
  L->o_nused = take(4 * L->chunk);
  L->o_Bp = take(4 * L->chunk);
  L->o_flags = take(4 * L->chunk);
  L->o_dirty = take(4 * L->chunk);
  L->o_ndirty = take(4);
  L->o_rec = take(L->rec_bytes);
  L->o_Mo = take(L->Mo_bytes);
  L->o_queue = take(8 * (kMaxDPGroups + 1));
  L->o_dpscr = take(L->dpscr_bytes);
  L->o_count = take(8 * n_pairs);
  L->o_order = take(4 * n_pairs);
  L->o_nf = L->o_perm = L->o_pos = L->o_grp = L->o_gstart = L->o_ngroups = L->o_nslot = -1;
  L->o_bounds = L->o_yhat = -1;
  L->o_hvars = L->o_hpairs = L->o_hscores = L->o_hM = -1;
  L->total = o;
  return GMINE_OK;
}

// Relative DP work of a pair with n samples and this B: per row count y the
// recursion over k <= min(c x, n) superclumps for x = floor(B / y) columns,
// both orientations alike (the sort key of the chunk planner).
double pair_cost(int n, int B, double c) {
  if (n < 4 || B < 4) return 0.0;
  double w = 0.0;
  for (int y = 2; y <= B / 2; ++y) {
    const double x = B / y;
    const double k = std::min<double>(host_khat(B, y, c), n);
    w += (x - 1.0) * k * k * 0.5 + k * k * 0.5 * y;
  }
  return w;
}

// The chunk's working arrays inside the uneven layout's regions, for C pairs
// of at most n samples and B <= Bc.
ChunkMem uneven_mem(void* ws, const Layout& L, int64_t C, int64_t n, int B) {
  ChunkMem cm{};
  const int64_t S = 2 * C;
  int64_t o = L.o_rank;
  auto sub = [&](int64_t bytes) { const int64_t at = o; o += align256(bytes); return at; };
  cm.rk.perm = at<int32_t>(ws, sub(4 * S * n));
  cm.rk.pos = at<int32_t>(ws, sub(4 * S * n));
  cm.rk.grp = at<int32_t>(ws, sub(4 * S * n));
  cm.rk.gstart = at<int32_t>(ws, sub(4 * S * (n + 1)));
  cm.rk.ngroups = at<int32_t>(ws, sub(4 * S));
  cm.rk.nslot = at<int32_t>(ws, sub(4 * S));
  cm.rk.stride = n;
  const int R = std::max(B / 2 - 1, 1);
  o = L.o_equi;
  cm.eq.bounds = at<int32_t>(ws, sub(4 * S * (int64_t)R * (R + 2)));
  cm.eq.yhat = at<int32_t>(ws, sub(4 * S * (int64_t)R));
  cm.eq.R = R;
  cm.eq.bstride = std::max(B / 2 - 1, 0) + 2;
  cm.pp = pair_prep(ws, L);
  cm.pp.order = at<int32_t>(ws, L.o_order);
  cm.rec = at<int32_t>(ws, L.o_rec);
  cm.Mo = at<double>(ws, L.o_Mo);
  cm.rec_off = at<int64_t>(ws, L.o_recoff);
  cm.queue = at<unsigned long long>(ws, L.o_queue);
  cm.partscr = L.o_partscr >= 0 ? at<unsigned char>(ws, L.o_partscr) : nullptr;
  cm.partscr_bytes = L.partscr_bytes;
  cm.rankscr = L.o_rankscr >= 0 ? at<unsigned char>(ws, L.o_rankscr) : nullptr;
  cm.rankscr_bytes = L.rankscr_bytes;
  cm.dpscr = at<char>(ws, L.o_dpscr);
  cm.dpscr_bytes = L.dpscr_bytes;
  return cm;
}

}  // namespace

namespace gm {
void note_cuda_error(cudaError_t e) { last_cuda_error() = e; }

cudaError_t allow_dynamic_smem(const void* func, int smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& have = granted[{func, dev}];
  if (smem <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) have = smem;
  return e;
}
}  // namespace gm

extern "C" {

int gmine_abi_version(void) { return GMINE_ABI_VERSION; }

int gmine_check_param(const gmine_param* param) {
  if (!param) return GMINE_E_ARG;
  if (!(param->alpha > 0.0 && param->alpha <= 1.0)) return GMINE_E_PARAM;
  if (!(param->c > 0.0) || !std::isfinite(param->c)) return GMINE_E_PARAM;
  return GMINE_OK;
}

const char* gmine_strerror(int status) {
  switch (status) {
    case GMINE_OK: return "ok";
    case GMINE_E_PARAM: return "invalid parameters: need 0 < alpha <= 1 and finite c > 0";
    case GMINE_E_TOO_FEW: return "too few usable samples (need n >= 4 and B >= 4)";
    case GMINE_E_CONSTANT: return "a variable is constant on the used samples";
    case GMINE_E_NOMEM: return "allocation failed";
    case GMINE_E_ARG: return "invalid argument";
    case GMINE_E_WORKSPACE: return "workspace smaller than gmine_plan reported";
    case GMINE_E_CUDA: return cudaGetErrorString(last_cuda_error());
    case GMINE_E_LIMIT: return "size beyond the limits of this build";
    case GMINE_E_NODEVICE: return "no usable CUDA device";
    case GMINE_E_TIMEOUT: return "a bounded wait inside a kernel ran out";
    default: return "unknown status";
  }
}

int gmine_B(int64_t n, double alpha) { return n > 0 ? host_B(n, alpha) : 0; }

int64_t gmine_m_cells(int32_t B) { return host_cells(B); }

int gmine_dp_groups(int64_t n, double alpha, double c, int32_t precision, gmine_dp_choice* out,
                    int32_t cap, int32_t* count) {
  if (!count || (cap > 0 && !out) || n < 0) return GMINE_E_ARG;
  const gmine_param prm{alpha, c};
  if (gmine_check_param(&prm) != GMINE_OK) return GMINE_E_PARAM;
  if (precision != GMINE_PLAIN_FP64 && precision != GMINE_FP32_DP_FP64_RESCORE) return GMINE_E_ARG;
  if (n > kMaxN) return GMINE_E_LIMIT;
  DeviceInfo dev;
  int rc = device_info(&dev);
  if (rc != GMINE_OK) return rc;
  ChunkPlan cp;
  rc = plan_chunk(n, n > 0 ? host_B(n, alpha) : 0, c, precision == GMINE_FP32_DP_FP64_RESCORE, dev, &cp);
  if (rc != GMINE_OK) return rc;
  *count = cp.ngroups;
  for (int gi = 0; gi < cp.ngroups && gi < cap; ++gi) {
    const DPGroup& g = cp.grp[gi];
    out[gi] = gmine_dp_choice{g.ylo, g.yhi, group_kind(g), g.threads, group_smem(g), g.lev};
  }
  return GMINE_OK;
}

int gmine_set_dp_choices(int64_t n, double alpha, double c, int32_t precision,
                         const gmine_dp_choice* choices, int32_t count) {
  if (n < 0 || count < 0 || (count > 0 && !choices) || count > kMaxDPGroups) return GMINE_E_ARG;
  const gmine_param prm{alpha, c};
  if (gmine_check_param(&prm) != GMINE_OK) return GMINE_E_PARAM;
  if (precision != GMINE_PLAIN_FP64 && precision != GMINE_FP32_DP_FP64_RESCORE) return GMINE_E_ARG;
  for (int i = 0; i < count; ++i)
    if (choices[i].kind < GMINE_DP_BLOCKED || choices[i].kind > GMINE_DP_TWO || choices[i].threads < 0 ||
        choices[i].ylo < 2 || choices[i].yhi < choices[i].ylo)
      return GMINE_E_ARG;
  const int B = n > 0 ? host_B(n, alpha) : 0;
  const bool fp32 = precision == GMINE_FP32_DP_FP64_RESCORE;
  std::lock_guard<std::mutex> lock(g_choice_mu);
  for (size_t i = 0; i < g_choice_sets.size(); ++i)
    if (g_choice_sets[i].n == n && g_choice_sets[i].B == B && g_choice_sets[i].c == c &&
        g_choice_sets[i].fp32 == fp32) {
      g_choice_sets.erase(g_choice_sets.begin() + (long)i);
      break;
    }
  if (count > 0)
    g_choice_sets.push_back(ChoiceSet{n, B, c, fp32, std::vector<gmine_dp_choice>(choices, choices + count)});
  return GMINE_OK;
}

int gmine_plan(int64_t p, int64_t n, int64_t n_pairs, const gmine_param* param, int32_t precision,
               int32_t flags, int64_t* m_cells_per_pair, int64_t* workspace_bytes) {
  Layout L;
  const int rc = make_layout(p, n, n_pairs, param, precision, flags, &L);
  if (rc != GMINE_OK) return rc;
  if (m_cells_per_pair) *m_cells_per_pair = L.cp.cells;
  if (workspace_bytes) *workspace_bytes = L.total;
  return GMINE_OK;
}

int gmine_compute_batch_ex(const double* d_vars, int64_t p, int64_t n, const int32_t* d_pairs,
                           int64_t n_pairs, const gmine_param* param, int32_t precision,
                           void* d_workspace, int64_t workspace_bytes, gmine_pair_score* d_scores,
                           double* d_M, const gmine_trace* trace, void* stream) {
  if (n_pairs > 0 && (!plausible_device_ptr(d_vars) || !d_pairs || !d_scores)) return GMINE_E_ARG;
  if (!d_workspace) return GMINE_E_ARG;
  const int32_t flags = trace ? GMINE_PLAN_TRACE : 0;
  Layout L;
  int rc = make_layout(p, n, n_pairs, param, precision, flags, &L);
  if (rc != GMINE_OK) return rc;
  if (workspace_bytes < L.total) return GMINE_E_WORKSPACE;
  if (n_pairs == 0) return GMINE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = d_workspace;
  int launches = 0;
  StageTiming stg;
  StageTiming* stages = (trace && trace->h_stage_ms) ? &stg : nullptr;
  if (stages) GM_CUDA(stages->mark(-1, st));
  rc = prepare_variables(d_vars, ws, L, param->alpha, param->c, st, &launches);
  if (rc != GMINE_OK) return rc;
  if (stages) GM_CUDA(stages->mark(GMINE_STAGE_SETUP, st));
  if (trace && trace->d_counters) GM_CUDA(cudaMemsetAsync(trace->d_counters, 0, 16, st));
  DPTiming tim;
  BatchCtx b{};
  b.vars = d_vars;
  b.p = p;
  b.n_row = n;
  b.pairs = d_pairs;
  b.n_pairs = n_pairs;
  b.c = param->c;
  b.fp32 = precision == GMINE_FP32_DP_FP64_RESCORE;
  b.ws = ws;
  b.L = &L;
  b.Btab = at<int32_t>(ws, L.o_Btab);
  b.Btab_slots = b.Btab;
  b.nf = at<int32_t>(ws, L.o_nf);
  b.scores = d_scores;
  b.M = d_M;
  b.m_stride = L.cp.cells;
  b.trace = trace;
  b.timing = (trace && trace->h_dp_ms) ? &tim : nullptr;
  b.stages = stages;
  b.st = st;
  b.launches = launches;
  const ChunkMem cm = regular_mem(ws, L);
  for (int64_t pair0 = 0; pair0 < n_pairs; pair0 += L.chunk) {
    rc = run_chunk(b, L.cp, cm, pair0, std::min(L.chunk, n_pairs - pair0));
    if (rc != GMINE_OK) return rc;
  }
  return finish_trace(b);
}

int gmine_compute_batch(const double* d_vars, int64_t p, int64_t n, const int32_t* d_pairs,
                        int64_t n_pairs, const gmine_param* param, int32_t precision,
                        void* d_workspace, int64_t workspace_bytes, gmine_pair_score* d_scores,
                        double* d_M, void* stream) {
  return gmine_compute_batch_ex(d_vars, p, n, d_pairs, n_pairs, param, precision, d_workspace,
                                workspace_bytes, d_scores, d_M, nullptr, stream);
}

int gmine_plan_uneven(int64_t p, int64_t n, int64_t n_pairs, const double* h_alphas,
                      int32_t n_alphas, double c, int32_t precision, int64_t* m_cells_per_pair,
                      int64_t* workspace_bytes) {
  Layout L;
  const int rc = make_layout_uneven(p, n, n_pairs, h_alphas, n_alphas, c, precision, &L);
  if (rc != GMINE_OK) return rc;
  if (m_cells_per_pair) *m_cells_per_pair = L.cp.cells;
  if (workspace_bytes) *workspace_bytes = L.total;
  return GMINE_OK;
}

int gmine_compute_batch_uneven(const double* d_vars, int64_t p, int64_t n, const int32_t* d_pairs,
                               int64_t n_pairs, const double* h_alphas, int32_t n_alphas,
                               const uint8_t* d_alpha_idx, double c, int32_t precision,
                               void* d_workspace, int64_t workspace_bytes,
                               gmine_pair_score* d_scores, double* d_M, const gmine_trace* trace,
                               void* stream) {
  if (n_pairs > 0 && (!plausible_device_ptr(d_vars) || !d_pairs || !d_scores)) return GMINE_E_ARG;
  if (!d_workspace) return GMINE_E_ARG;
  if (n_alphas > 1 && !d_alpha_idx) return GMINE_E_ARG;
  if (trace && (trace->d_k || trace->d_yhat || trace->d_clumps || trace->d_sc_ends ||
                trace->d_cuts || trace->d_I))
    return GMINE_E_ARG;  // per-task outputs follow the batch order: not here
  Layout L;
  int rc = make_layout_uneven(p, n, n_pairs, h_alphas, n_alphas, c, precision, &L);
  if (rc != GMINE_OK) return rc;
  if (workspace_bytes < L.total) return GMINE_E_WORKSPACE;
  if (n_pairs == 0) return GMINE_OK;
  DeviceInfo dev;
  rc = device_info(&dev);
  if (rc != GMINE_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = d_workspace;
  const bool fp32 = precision == GMINE_FP32_DP_FP64_RESCORE;
  // the pairs' alpha indices are checked on the host before any table is
  // read through them
  if (d_alpha_idx) {
    std::vector<uint8_t> ai((size_t)n_pairs);
    GM_CUDA(cudaMemcpyAsync(ai.data(), d_alpha_idx, (size_t)n_pairs, cudaMemcpyDeviceToHost, st));
    GM_CUDA(cudaStreamSynchronize(st));
    for (uint8_t a : ai)
      if (a >= n_alphas) return GMINE_E_ARG;
  }
  StageTiming stg;
  StageTiming* stages = (trace && trace->h_stage_ms) ? &stg : nullptr;
  if (stages) GM_CUDA(stages->mark(-1, st));
  rc = upload_Btab(ws, L, h_alphas, n_alphas, st);
  if (rc != GMINE_OK) return rc;
  int launches = 0;
  const int32_t* Btab = at<int32_t>(ws, L.o_Btab);
  k_tables<<<(unsigned)((n + 256) / 256), 256, 0, st>>>((int)n, at<double>(ws, L.o_L64),
                                                        at<float>(ws, L.o_L32), at<double>(ws, L.o_lnt),
                                                        L.cp.B, (int)n, c, at<int64_t>(ws, L.o_recoff));
  GM_CUDA(cudaGetLastError());
  ++launches;
  // samples used and B of every pair, read back to plan the chunks
  int32_t* cnt_d = at<int32_t>(ws, L.o_count);
  k_pair_count<<<(unsigned)((n_pairs + 7) / 8), 256, 0, st>>>(d_vars, p, n, d_pairs, n_pairs,
                                                              d_alpha_idx, Btab, n + 1, cnt_d);
  GM_CUDA(cudaGetLastError());
  ++launches;
  std::vector<int32_t> cnt((size_t)(2 * n_pairs));
  GM_CUDA(cudaMemcpyAsync(cnt.data(), cnt_d, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  // heaviest pairs first, so that each chunk holds pairs of similar size
  std::vector<double> cost((size_t)n_pairs);
  for (int64_t i = 0; i < n_pairs; ++i) cost[i] = pair_cost(cnt[2 * i], cnt[2 * i + 1], c);
  std::vector<int32_t> order((size_t)n_pairs);
  for (int64_t i = 0; i < n_pairs; ++i) order[i] = (int32_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  GM_CUDA(cudaMemcpyAsync(at<int32_t>(ws, L.o_order), order.data(), sizeof(int32_t) * order.size(),
                          cudaMemcpyHostToDevice, st));
  if (stages) GM_CUDA(stages->mark(GMINE_STAGE_SETUP, st));
  if (trace && trace->d_counters) GM_CUDA(cudaMemsetAsync(trace->d_counters, 0, 16, st));
  DPTiming tim;
  BatchCtx b{};
  b.vars = d_vars;
  b.p = p;
  b.n_row = n;
  b.pairs = d_pairs;
  b.n_pairs = n_pairs;
  b.c = c;
  b.fp32 = fp32;
  b.ws = ws;
  b.L = &L;
  b.Btab = Btab;
  b.Btab_slots = Btab + (int64_t)n_alphas * (n + 1);
  b.nf = nullptr;
  b.scores = d_scores;
  b.M = d_M;
  b.m_stride = L.cp.cells;
  b.trace = trace;
  b.timing = (trace && trace->h_dp_ms) ? &tim : nullptr;
  b.stages = stages;
  b.st = st;
  b.launches = launches;
  int64_t i = 0;
  while (i < n_pairs) {
    // the longest run of pairs (in cost order) whose chunk fits every region
    int64_t j = i, nc = 4;
    int Bc = 0;
    while (j < n_pairs && j - i < L.chunk) {
      const int32_t q = order[j];
      const int64_t n2 = std::max<int64_t>(nc, cnt[2 * q]);
      const int B2 = std::max(Bc, cnt[2 * q + 1]);
      const ChunkBytes cb = chunk_bytes(j - i + 1, n2, B2, c);
      if (cb.rank > L.rank_bytes || cb.equi > L.equi_bytes || cb.rec > L.rec_bytes ||
          cb.Mo > L.Mo_bytes) {
        if (j == i) return GMINE_E_LIMIT;
        break;
      }
      nc = n2;
      Bc = B2;
      ++j;
    }
    ChunkPlan cp;
    rc = plan_chunk(nc, Bc, c, fp32, dev, &cp);
    if (rc != GMINE_OK) return rc;
    ChunkMem cm = uneven_mem(ws, L, j - i, nc, Bc);
    cm.pp.aidx = d_alpha_idx;
    if (stages) GM_CUDA(stages->mark(-1, st));
    k_tables<<<1, 256, 0, st>>>(-1, nullptr, nullptr, nullptr, Bc, (int)nc, c, cm.rec_off);
    GM_CUDA(cudaGetLastError());
    ++b.launches;
    if (stages) GM_CUDA(stages->mark(GMINE_STAGE_SETUP, st));
    rc = run_chunk(b, cp, cm, i, j - i);
    if (rc != GMINE_OK) return rc;
    i = j;
  }
  return finish_trace(b);
}

int gmine_compute_batch_host(const double* h_vars, int64_t p, int64_t n, const int32_t* h_pairs,
                             int64_t n_pairs, const gmine_param* param, int32_t precision,
                             void* d_workspace, int64_t workspace_bytes,
                             gmine_pair_score* h_scores, double* h_M, void* stream) {
  if (n_pairs > 0 && (!h_vars || !h_pairs || !h_scores)) return GMINE_E_ARG;
  if (!d_workspace) return GMINE_E_ARG;
  Layout L;
  int rc = make_layout(p, n, n_pairs, param, precision, GMINE_PLAN_HOST_STAGING, &L);
  if (rc != GMINE_OK) return rc;
  if (workspace_bytes < L.total) return GMINE_E_WORKSPACE;
  if (n_pairs == 0) return GMINE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* dv = at<double>(d_workspace, L.o_hvars);
  int32_t* dp = at<int32_t>(d_workspace, L.o_hpairs);
  gmine_pair_score* ds = at<gmine_pair_score>(d_workspace, L.o_hscores);
  double* dM = h_M ? at<double>(d_workspace, L.o_hM) : nullptr;
  GM_CUDA(cudaMemcpyAsync(dv, h_vars, 8 * p * n, cudaMemcpyHostToDevice, st));
  GM_CUDA(cudaMemcpyAsync(dp, h_pairs, 8 * n_pairs, cudaMemcpyHostToDevice, st));
  rc = gmine_compute_batch(dv, p, n, dp, n_pairs, param, precision, d_workspace, workspace_bytes,
                           ds, dM, stream);
  if (rc != GMINE_OK) return rc;
  GM_CUDA(cudaMemcpyAsync(h_scores, ds, sizeof(gmine_pair_score) * n_pairs,
                          cudaMemcpyDeviceToHost, st));
  if (h_M) GM_CUDA(cudaMemcpyAsync(h_M, dM, 8 * n_pairs * L.cp.cells, cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  return GMINE_OK;
}

int gmine_rank(const double* d_vars, int64_t p, int64_t n, int32_t* d_perm, int32_t* d_rank,
               int32_t* d_groups, void* d_workspace, int64_t workspace_bytes, void* stream) {
  if (!d_vars || !d_perm || !d_rank || !d_groups || !d_workspace) return GMINE_E_ARG;
  gmine_param prm{0.6, 15.0};
  Layout L;
  int rc = make_layout(p, n, 0, &prm, GMINE_PLAIN_FP64, 0, &L);
  if (rc != GMINE_OK) return rc;
  if (workspace_bytes < L.total) return GMINE_E_WORKSPACE;
  if (p == 0 || n == 0) return GMINE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int launches = 0;
  rc = prepare_variables(d_vars, d_workspace, L, prm.alpha, prm.c, st, &launches);
  if (rc != GMINE_OK) return rc;
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)p);
  k_rank_export<<<grid, 256, 0, st>>>(rank_data(d_workspace, L), p, d_rank, d_perm, d_groups);
  GM_CUDA(cudaGetLastError());
  return GMINE_OK;
}

int gmine_equipartition(const double* d_vars, int64_t p, int64_t n, int32_t y, int32_t* d_Q,
                        int32_t* d_yhat, void* d_workspace, int64_t workspace_bytes,
                        void* stream) {
  if (!d_vars || !d_Q || !d_yhat || !d_workspace || y < 1) return GMINE_E_ARG;
  gmine_param prm{0.6, 15.0};
  Layout L;
  int rc = make_layout(p, n, 0, &prm, GMINE_PLAIN_FP64, 0, &L);
  if (rc != GMINE_OK) return rc;
  if (workspace_bytes < L.total) return GMINE_E_WORKSPACE;
  if (p == 0 || n == 0) return GMINE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int launches = 0;
  rc = prepare_variables(d_vars, d_workspace, L, prm.alpha, prm.c, st, &launches);
  if (rc != GMINE_OK) return rc;
  // one row count y for every variable: reuse the bounds rows of y = 2
  // as output space through a dedicated single-y kernel
  EquiData eq1;
  eq1.bounds = at<int32_t>(d_workspace, L.o_bounds);
  eq1.yhat = at<int32_t>(d_workspace, L.o_yhat);
  eq1.R = 1;
  eq1.bstride = y + 1;
  if ((int64_t)p * (y + 1) > (int64_t)L.slots * L.cp.R * L.cp.bstride)
    return GMINE_E_LIMIT;
  k_equi_single<<<(unsigned)((p + 127) / 128), 128, 0, st>>>(p, y, rank_data(d_workspace, L), eq1);
  GM_CUDA(cudaGetLastError());
  dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)p);
  k_equi_export<<<grid, 256, 0, st>>>(rank_data(d_workspace, L), eq1, p, 2, d_Q, d_yhat);
  GM_CUDA(cudaGetLastError());
  return GMINE_OK;
}

int gmine_pearson_batch(const double* d_vars, int64_t p, int64_t n, const int32_t* d_pairs,
                        int64_t n_pairs, const gmine_pair_score* d_scores, double* d_rho,
                        double* d_nonlin, void* stream) {
  if (p < 0 || n < 0 || n_pairs < 0) return GMINE_E_ARG;
  if (n_pairs == 0) return GMINE_OK;
  if (!plausible_device_ptr(d_vars) || !d_pairs || !d_rho) return GMINE_E_ARG;
  if (d_nonlin && !d_scores) return GMINE_E_ARG;
  DeviceInfo dev;
  const int rc = device_info(&dev);
  if (rc != GMINE_OK) return rc;
  // eight 256-thread CTAs (64 warps, one pair each) per SM, grid-stride
  const int64_t grid = std::min<int64_t>((n_pairs + 7) / 8, (int64_t)dev.sms * 8);
  GM_CUDA(pearson_launch((int)grid, static_cast<cudaStream_t>(stream), d_vars, p, n, d_pairs,
                         n_pairs, d_scores, d_rho, d_nonlin));
  return GMINE_OK;
}

int gmine_score_pair_host(const double* h_x, const double* h_y, int64_t n,
                          const gmine_param* param, int32_t precision, gmine_pair_score* out,
                          double* M_out) {
  if (!h_x || !h_y || !out || n < 0) return GMINE_E_ARG;
  int64_t cells = 0, wsb = 0;
  int rc = gmine_plan(2, n, 1, param, precision, GMINE_PLAN_HOST_STAGING, &cells, &wsb);
  if (rc != GMINE_OK) return rc;
  std::vector<double> vars((size_t)(2 * n));
  if (n > 0) {
    std::memcpy(vars.data(), h_x, sizeof(double) * n);
    std::memcpy(vars.data() + n, h_y, sizeof(double) * n);
  }
  const int32_t pairs[2] = {0, 1};
  void* ws = nullptr;
  if (cudaMalloc(&ws, (size_t)wsb) != cudaSuccess) return GMINE_E_NOMEM;
  std::vector<double> M((size_t)std::max<int64_t>(cells, 1));
  rc = gmine_compute_batch_host(vars.data(), 2, n, pairs, 1, param, precision, ws, wsb, out,
                                M.data(), nullptr);
  cudaFree(ws);
  if (rc == GMINE_OK && M_out) std::memcpy(M_out, M.data(), sizeof(double) * out->m_cells);
  return rc;
}

double gmine_mic(const gmine_pair_score* s) { return s ? s->mic : 0.0; }
double gmine_mas(const gmine_pair_score* s) { return s ? s->mas : 0.0; }
double gmine_mev(const gmine_pair_score* s) { return s ? s->mev : 0.0; }
double gmine_mcn(const gmine_pair_score* s) { return s ? s->mcn : 0.0; }

}  // extern "C"
