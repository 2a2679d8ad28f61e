/*
 * gmine.h -- C ABI of libgmine, the GB300 (sm_103a) implementation of the
 * MINE statistics over many variable pairs.
 *
 * The calls follow the problem statement of the C engine the paper describes
 * (Sec. "The MINE C engine and its wrappers"): a dataset of variables, a
 * parameter structure {alpha, c}, and per pair a score structure holding the
 * characteristic matrix M and the four statistics MIC, MAS, MEV, MCN.
 *
 * Definitions implemented (the method's steps, in the order the paper and the
 * SOM algorithms it refers to give them):
 *   B = floor(n^alpha) with n the samples left after dropping missing ones
 *     (Sec. 2C: B(n) = n^alpha);
 *   for both orientations and every row count y = 2..floor(B/2):
 *     EquipartitionYAxis of the row variable (Appendix items 3-4),
 *     GetClumpsPartition / GetSuperclumpsPartition of the column variable
 *     with khat = floor(c * floor(B/y)) (Appendix items 5-7, the two
 *     algorithm listings), and the OptimizeXAxis dynamic program over the
 *     superclumps with precomputed cell counts and entropy terms (Appendix
 *     item 10), giving I(x, y) for x = 2..floor(B/y);
 *   M(x,y) = I / log min(x, yhat), the larger of the two orientations,
 *     over x*y <= B (Appendix items 1 and 4);
 *   MIC = max M; MAS = max |M(x,y) - M(y,x)|; MEV = max M over x = 2 or
 *     y = 2; MCN = min log2(xy) over the cells with M = MIC (Appendix item 2).
 *
 * Conventions for every call:
 *   - Pointers named d_* are CUDA device pointers, h_* host pointers.  The
 *     caller owns every buffer; the library keeps no pointer after a call
 *     returns.  Except for gmine_score_pair_host, no call allocates device
 *     memory: gmine_plan reports the workspace the caller must provide.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls taking d_* pointers only enqueue work on it and
 *     return; results are ready once the stream has been synchronised.
 *     The batch calls also copy a small table (B(m) = floor(m^alpha), made
 *     with the host's pow) from host memory with cudaMemcpyAsync on it.
 *   - Several host threads may call the library at once, each with its own
 *     workspace and stream: the shared-memory limits the calls set on the
 *     kernels only ever grow, so one call's planning never lowers what
 *     another call's launches need.
 *   - Every call returns an int status (GMINE_OK = 0 or a GMINE_E_* code);
 *     nothing aborts or throws across this boundary.  A per-pair status is
 *     also stored in each gmine_pair_score.
 *   - Variables are stored variable-major: d_vars[v * n + i] is sample i of
 *     variable v (one variable per row, as in the paper's data files).  A
 *     sample that is NaN or infinite is missing; a pair uses the samples
 *     where both of its variables are finite.
 *   - Pairs are int32 [n_pairs][2]: (index of X, index of Y).  In the score
 *     of a pair, M(x, y) has x columns on X and y rows on Y.
 */
#ifndef GMINE_H
#define GMINE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMINE_ABI_VERSION 3

/* status codes */
#define GMINE_OK 0
#define GMINE_E_PARAM 1      /* alpha not in (0, 1] or c not finite and > 0 */
#define GMINE_E_TOO_FEW 2    /* pair: fewer than 4 usable samples or B < 4 */
#define GMINE_E_CONSTANT 3   /* pair: a variable is constant on the used
                                samples; that orientation contributes M = 0 */
#define GMINE_E_NOMEM 4      /* host or device allocation failed */
#define GMINE_E_ARG 5        /* NULL pointer, negative size, bad index */
#define GMINE_E_WORKSPACE 6  /* workspace smaller than gmine_plan reported */
#define GMINE_E_CUDA 7       /* a CUDA runtime call failed */
#define GMINE_E_LIMIT 8      /* a size beyond what this build supports (n > 131072) */
#define GMINE_E_NODEVICE 9   /* no usable CUDA device */
#define GMINE_E_TIMEOUT 10   /* pair: a bounded wait between the warps of a
                                kernel ran out; the pair's results are not
                                valid (not expected: a safety bound) */

/* precision of the OptimizeXAxis dynamic program */
#define GMINE_PLAIN_FP64 0            /* entropies and DP in double */
#define GMINE_FP32_DP_FP64_RESCORE 1  /* DP in float with exact int32 counts;
                                         each chosen partition re-scored in
                                         double */

/* Parameters (Sec. "The MINE C engine": the configuration structure).
   alpha: B = n^alpha, 0 < alpha <= 1 (paper default 0.6);
   c: clump factor, khat = c * x, c > 0 (paper default 15). */
typedef struct {
    double alpha;
    double c;
} gmine_param;

/* Score of one pair (72 bytes). */
typedef struct {
    double mic, mas, mev, mcn;
    int64_t m_offset;   /* first cell of this pair in d_M / h_M           */
    int32_t n_used;     /* samples where both variables are finite        */
    int32_t B;          /* floor(n_used^alpha)                            */
    int32_t m_cells;    /* cells (x, y), x, y >= 2, x*y <= B, y-major     */
    int32_t mcn_xy;     /* the x*y whose log2 is MCN                      */
    int32_t status;     /* GMINE_OK, GMINE_E_TOO_FEW, GMINE_E_CONSTANT, or
                           GMINE_E_ARG for a pair index outside [0, p)    */
    int32_t yhat_x;     /* rows used when X is equipartitioned into 2     */
    int32_t yhat_y;     /* rows used when Y is equipartitioned into 2     */
    int32_t reserved;
} gmine_pair_score;

/* Optional per-task outputs of gmine_compute_batch_ex, for parity checks of
   the integer quantities.  A task is (pair, orientation o, row count y):
   o = 0 equipartitions Y and optimises columns on X, o = 1 the reverse.
   Task t of the batch is  t = ((y - 2) * 2 + o) * n_pairs + pair  for
   y = 2 .. floor(B_max/2), B_max = floor(n^alpha) of the full sample count.
   Every pointer may be NULL.  Strides are in elements. */
typedef struct {
    int32_t *d_k;         /* [tasks] superclumps k (0 if task is empty)    */
    int32_t *d_yhat;      /* [tasks] rows used                              */
    int32_t *d_clumps;    /* [tasks] clumps before the superclump step      */
    int32_t *d_sc_ends;   /* [tasks][sc_stride] superclump ends c_0..c_k    */
    int32_t sc_stride;
    int32_t cut_stride;
    int32_t *d_cuts;      /* [tasks][cut_stride] chosen partition of each
                             l = 2..x: its l-1 column ends (superclump
                             indices) packed at (l-2)(l-1)/2; -1 where l > k */
    double *d_I;          /* [tasks][I_stride] I(l) for l = 2..x            */
    int32_t I_stride;
    int32_t reserved;
    int64_t *d_counters;  /* [2] device: subtract-and-max steps of the DP and
                             tasks run; zeroed by the call                  */
    double *h_dp_ms;      /* host: if not NULL the call times each launch of
                             the DP kernel with CUDA events on `stream`,
                             synchronises the stream before returning, and
                             stores the summed milliseconds here           */
    int32_t *h_dp_launches;  /* host: number of DP kernel launches timed   */
    int32_t *h_kernel_launches;  /* host: if not NULL, every kernel launch of
                                    the call is counted here               */
    float *h_launch_ms;   /* host: with h_dp_ms, the milliseconds of each DP
                             launch in launch order (chunks, then launch
                             groups as gmine_dp_groups lists them), at most
                             launch_cap of them                            */
    int32_t launch_cap;
    int32_t reserved2;
    double *h_stage_ms;   /* host: if not NULL, [GMINE_N_STAGES] milliseconds
                             of each stage of the call (GMINE_STAGE_*), summed
                             over chunks, from CUDA events recorded on
                             `stream` between the stages; the stream is
                             synchronised before returning.  The call's
                             stream time outside these intervals (host work
                             between chunks, event gaps) is in none.      */
} gmine_trace;

/* Stages of a batch call, indexes of gmine_trace.h_stage_ms. */
#define GMINE_STAGE_SETUP 0      /* per-variable preparation: non-finite counts,
                                    ranks, equipartitions, L and log tables;
                                    for uneven batches the pair sizes and the
                                    chunk tables */
#define GMINE_STAGE_PAIRS 1      /* per chunk: pair slots and per-pair ranks */
#define GMINE_STAGE_EQUI 2       /* per chunk: per-pair equipartitions */
#define GMINE_STAGE_PARTITION 3  /* per chunk: clumps, superclumps, count
                                    tables of every task */
#define GMINE_STAGE_DP 4         /* per chunk: the OptimizeXAxis launches */
#define GMINE_STAGE_FINAL 5      /* per chunk: M and the statistics */
#define GMINE_N_STAGES 6

/* ---- parameters, errors ------------------------------------------------ */

int gmine_abi_version(void);

/* GMINE_OK if 0 < alpha <= 1 and c is finite and > 0, else GMINE_E_PARAM
   (the C++ wrapper of the paper rejects invalid parameters). */
int gmine_check_param(const gmine_param *param);

/* Static English text for a status code. */
const char *gmine_strerror(int status);

/* B = floor(n^alpha) as the library computes it (double pow on the host). */
int gmine_B(int64_t n, double alpha);

/* Number of cells of M for a given B. */
int64_t gmine_m_cells(int32_t B);

/* ---- kernel choices of the dynamic program (autotuning) ---------------- */

/* Kernel shapes of the OptimizeXAxis launches (Appendix item 10; SOM Alg. 2). */
#define GMINE_DP_BLOCKED 0  /* CTA per task, t in blocks of 32, levels in registers */
#define GMINE_DP_WARP 1     /* warp per task, the same blocked recursion (float only) */
#define GMINE_DP_MID 2      /* CTA per task, level after level, entropy triangle in
                               shared memory (8-12 levels) */
#define GMINE_DP_SMALL 3    /* warp per task, level after level (x <= 5) */
#define GMINE_DP_TWO 4      /* x = 2: two entropy terms per candidate */

/* One launch group of the DP: the tasks with row counts y in [ylo, yhi],
   its kernel shape and CTA size (threads); smem and lev are outputs of
   gmine_dp_groups (dynamic shared memory per CTA, levels per pass). */
typedef struct {
    int32_t ylo, yhi;
    int32_t kind;
    int32_t threads;
    int32_t smem;
    int32_t lev;
} gmine_dp_choice;

/* The launch groups the planner makes on the current device for a batch
   of n samples with these parameters, with the kernel shape and CTA size
   each gets (the built-in rules, or a choice set by gmine_set_dp_choices
   when it is feasible).  Writes min(*count, cap) entries; *count = number
   of groups.  GMINE_E_ARG / GMINE_E_PARAM / GMINE_E_LIMIT as gmine_plan. */
int gmine_dp_groups(int64_t n, double alpha, double c, int32_t precision,
                    gmine_dp_choice *out, int32_t cap, int32_t *count);

/* Tuned choices for batches with these (n, alpha, c, precision): a choice
   replaces the built-in rule of the launch group with the same [ylo, yhi]
   whenever its kernel shape applies to the group and its shared-memory plan
   fits the device (else the rule stays).  count = 0 removes them.  The
   table is process-wide and read when a call is planned; gmine_dp_groups
   shows the effect.  GMINE_E_ARG for a bad kind, range or count. */
int gmine_set_dp_choices(int64_t n, double alpha, double c, int32_t precision,
                         const gmine_dp_choice *choices, int32_t count);

/* ---- batch over pairs -------------------------------------------------- */

/* flags for gmine_plan */
#define GMINE_PLAN_HOST_STAGING 1   /* workspace also holds device copies of
                                       the inputs and outputs, as needed by
                                       gmine_compute_batch_host */
#define GMINE_PLAN_TRACE 2          /* accepted for compatibility; the trace
                                       needs no extra workspace */

/* Sizes for a batch of n_pairs pairs over p variables of n samples.
   *m_cells_per_pair: cells of M reserved per pair (pair i's cells start at
   i * m_cells_per_pair in d_M).  *workspace_bytes: device workspace to pass
   to the compute calls (256-byte aligned).  Either output may be NULL. */
int gmine_plan(int64_t p, int64_t n, int64_t n_pairs, const gmine_param *param,
               int32_t precision, int32_t flags, int64_t *m_cells_per_pair,
               int64_t *workspace_bytes);

/* The characteristic matrix and statistics of every pair (the paper's
   mine_compute_score over a dataset).  d_vars [p][n] double, d_pairs
   [n_pairs][2] int32, d_scores [n_pairs], d_M [n_pairs * m_cells_per_pair]
   double or NULL.  Asynchronous on `stream`. */
int gmine_compute_batch(const double *d_vars, int64_t p, int64_t n,
                        const int32_t *d_pairs, int64_t n_pairs,
                        const gmine_param *param, int32_t precision,
                        void *d_workspace, int64_t workspace_bytes,
                        gmine_pair_score *d_scores, double *d_M, void *stream);

/* As gmine_compute_batch, plus the per-task outputs of `trace` (may be
   NULL; the workspace must then be planned with GMINE_PLAN_TRACE). */
int gmine_compute_batch_ex(const double *d_vars, int64_t p, int64_t n,
                           const int32_t *d_pairs, int64_t n_pairs,
                           const gmine_param *param, int32_t precision,
                           void *d_workspace, int64_t workspace_bytes,
                           gmine_pair_score *d_scores, double *d_M,
                           const gmine_trace *trace, void *stream);

/* Host buffers in and out: copies h_vars and h_pairs into the workspace
   (planned with GMINE_PLAN_HOST_STAGING), computes, copies the scores (and M
   if h_M is not NULL) back and synchronises `stream` before returning. */
int gmine_compute_batch_host(const double *h_vars, int64_t p, int64_t n,
                             const int32_t *h_pairs, int64_t n_pairs,
                             const gmine_param *param, int32_t precision,
                             void *d_workspace, int64_t workspace_bytes,
                             gmine_pair_score *h_scores, double *h_M,
                             void *stream);

/* ---- batches of uneven pairs ------------------------------------------- */

/* Largest number of distinct alpha values in one uneven batch. */
#define GMINE_MAX_ALPHAS 8

/* Sizes for gmine_compute_batch_uneven (same arguments as its call):
   *m_cells_per_pair: cells of M reserved per pair, those of
   B = floor(n^max alpha); *workspace_bytes: the workspace to pass (a few
   GB for large n and alpha: the records of a chunk of heavy pairs take up
   to 24 GiB).  Errors: GMINE_E_ARG (NULL h_alphas, n_alphas < 1, negative
   sizes), GMINE_E_PARAM (an alpha outside (0, 1] or c not finite and > 0),
   GMINE_E_LIMIT (n_alphas > GMINE_MAX_ALPHAS or n > 131072). */
int gmine_plan_uneven(int64_t p, int64_t n, int64_t n_pairs, const double *h_alphas,
                      int32_t n_alphas, double c, int32_t precision,
                      int64_t *m_cells_per_pair, int64_t *workspace_bytes);

/* mine_compute_score over pairs of uneven size, each with its own alpha:
   pair i uses the n_i samples where both its variables are finite and
   B_i = floor(n_i^alpha_i) (Sec. 2C: B(n) = n^alpha, per pair), with the
   same steps and kernels as gmine_compute_batch.
   - d_vars [p][n] double, shorter variables padded with NaN; d_pairs
     [n_pairs][2] int32; both device memory.
   - h_alphas: host array of the n_alphas distinct alpha values (1 ..
     GMINE_MAX_ALPHAS); d_alpha_idx: device uint8 [n_pairs], pair i takes
     h_alphas[d_alpha_idx[i]] (NULL allowed when n_alphas == 1).
   - d_scores [n_pairs] and d_M [n_pairs * m_cells_per_pair] (or NULL) as for
     gmine_compute_batch: pair i's score at i, its cells at i *
     m_cells_per_pair.
   - trace: NULL, or only the counters and timing fields set (d_counters,
     h_dp_ms, h_dp_launches, h_kernel_launches, h_launch_ms, h_stage_ms);
     per-task arrays are refused.
   How it runs: the pairs' alpha indices and sample counts are read back to
   the host (the call synchronises `stream` twice), the pairs are ordered by
   their DP work, heaviest first, and cut into chunks that fit the
   workspace, each planned for its own largest n and B; each pair gets its
   own compacted ranks.  A pair's result does not depend on the rest of
   the batch.  Returns once the last chunk is enqueued.
   Errors: GMINE_E_ARG (NULL pointers, an alpha index >= n_alphas, per-task
   trace arrays), GMINE_E_PARAM, GMINE_E_LIMIT as gmine_plan_uneven,
   GMINE_E_WORKSPACE, GMINE_E_CUDA; per-pair statuses as gmine_compute_batch. */
int gmine_compute_batch_uneven(const double *d_vars, int64_t p, int64_t n,
                               const int32_t *d_pairs, int64_t n_pairs,
                               const double *h_alphas, int32_t n_alphas,
                               const uint8_t *d_alpha_idx, double c, int32_t precision,
                               void *d_workspace, int64_t workspace_bytes,
                               gmine_pair_score *d_scores, double *d_M,
                               const gmine_trace *trace, void *stream);

/* ---- batch without a caller workspace ---------------------------------- */

/* gmine_compute_batch with the working memory taken from a fixed array
   inside the library (64 MiB per GPU) instead of a workspace from the
   caller.  The paper has no counterpart of this call.
   It serves callers that cannot allocate device memory: code hosted by an
   application that owns the GPU's memory through its own pool and does not
   let plug-ins call cudaMalloc, and code on a latency-critical path that
   cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
   The call allocates nothing.  Inputs and outputs are the caller's, exactly
   as for gmine_compute_batch (d_M may be NULL).
   - Limit: batches whose gmine_plan workspace exceeds 64 MiB are refused
     with GMINE_E_WORKSPACE before anything is enqueued (a few hundred pairs
     at n ~ 1000, or one pair up to a few thousand samples at alpha = 0.6).
   - The first call on each device looks up the array's device address
     (cudaGetSymbolAddress with that device current) and keeps it; make that
     first call before any stream capture.  A reset of the device
     (cudaDeviceReset) after that first call is not supported: the kept
     address would then be stale.
   - Every call on a device shares the one array.  Its contents from an
     earlier call do not matter (the computation initialises all it reads),
     but calls whose work can overlap on the GPU (other streams, other host
     threads) race on it: order them, e.g. on one stream.
   The array is device code of the library: with lazy module loading (the
   CUDA runtime's default) a device reserves its 64 MiB when this call first
   runs there; with CUDA_MODULE_LOADING=EAGER every device on which the
   process uses the CUDA runtime reserves it, whether or not the call runs.
   Either way it stays reserved until the process exits. */
int gmine_compute_batch_static(const double *d_vars, int64_t p, int64_t n,
                               const int32_t *d_pairs, int64_t n_pairs,
                               const gmine_param *param, int32_t precision,
                               gmine_pair_score *d_scores, double *d_M,
                               void *stream);

/* ---- the linear statistics reported beside MINE ------------------------ */

/* Pearson correlation and the non-linearity index of each listed pair: the
   paper's analyses report them next to the four MINE statistics (Fig. 1
   caption; SI Sec. 2A, "four MINE statistics, Pearson and non-linearity").
   - d_rho[i]: Pearson rho of pair i over the samples where both variables
     are finite (the same samples as its MINE score), the two-pass form
     S_xy / sqrt(S_xx * S_yy) in double; NaN when fewer than two samples
     remain, a variance is zero or a pair index is outside [0, p).
   - d_nonlin[i] (may be NULL): MIC - rho^2, the paper naming the index
     without a formula and this being its definition in the MINE statistics'
     original paper; needs d_scores from gmine_compute_batch* for the same
     pairs (NULL d_scores with non-NULL d_nonlin is GMINE_E_ARG).  NaN where
     rho is NaN or the pair's status is not GMINE_OK.
   Layouts as for gmine_compute_batch (d_vars [p][n], d_pairs [n_pairs][2]);
   all pointers are device pointers owned by the caller; asynchronous on
   `stream`; nothing is allocated.  Errors: GMINE_E_ARG for negative sizes or
   missing pointers, GMINE_E_CUDA if the launch fails. */
int gmine_pearson_batch(const double *d_vars, int64_t p, int64_t n,
                        const int32_t *d_pairs, int64_t n_pairs,
                        const gmine_pair_score *d_scores, double *d_rho,
                        double *d_nonlin, void *stream);

/* ---- single steps, the same kernels as the batch uses ------------------ */

/* Tie-aware sort of every variable (finite samples; no NaN allowed):
   d_perm[v][m] = sample at sorted position m (ties by sample index),
   d_rank[v][i] = dense rank of sample i (0 = smallest value),
   d_groups[v] = number of distinct values.  Workspace as gmine_plan(p, n,
   0, ...) reports.  GMINE_E_ARG if a variable holds a non-finite sample. */
int gmine_rank(const double *d_vars, int64_t p, int64_t n, int32_t *d_perm,
               int32_t *d_rank, int32_t *d_groups, void *d_workspace,
               int64_t workspace_bytes, void *stream);

/* EquipartitionYAxis (SOM Alg. 3; Appendix items 3-4) of every variable
   into y rows: d_Q[v][i] = 0-based row of sample i, d_yhat[v] = rows used. */
int gmine_equipartition(const double *d_vars, int64_t p, int64_t n, int32_t y,
                        int32_t *d_Q, int32_t *d_yhat, void *d_workspace,
                        int64_t workspace_bytes, void *stream);

/* ---- one pair, host memory (convenience; allocates and synchronises) --- */

/* mine_compute_score for one dataset of two variables x, y of n samples.
   M_out may be NULL, else it receives out->m_cells doubles. */
int gmine_score_pair_host(const double *h_x, const double *h_y, int64_t n,
                          const gmine_param *param, int32_t precision,
                          gmine_pair_score *out, double *M_out);

/* The four statistic functions of the paper's score structure. */
double gmine_mic(const gmine_pair_score *s);
double gmine_mas(const gmine_pair_score *s);
double gmine_mev(const gmine_pair_score *s);
double gmine_mcn(const gmine_pair_score *s);

#ifdef __cplusplus
}
#endif

#endif /* GMINE_H */
