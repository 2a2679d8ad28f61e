/*
 * mine_oracle.c -- plain, slow FP64 CPU oracle for the MINE characteristic
 * matrix and the MIC / MAS / MEV / MCN statistics (Albanese et al.,
 * "minerva and minepy: a C engine for the MINE suite", 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every function follows the method step by step, in the order in which the
 * paper (and the Reshef et al. 2011 SOM algorithms it refers to) states it.
 * No blocking, fusion or reordering beyond that.  Floating point is IEEE
 * double throughout (Appendix item 9); the build turns FP contraction off so
 * that every expression rounds exactly as written.
 *
 * Conventions: samples are 0-based; row labels (Q) and column labels (P) are
 * 0-based here (the paper's are 1-based).  "Sorted position" means the index
 * of a sample in the ascending order of a variable, ties broken by sample
 * index (any tie order gives the same results, see the comments below).
 *
 * Readings of points where the paper is silent or garbled (kept in the same
 * form in the design notes):
 *   R1 B = floor(pow(n, alpha)) in double (Sec. 2C states B(n) = n^alpha).
 *   R2 the domain is x*y <= B (Appendix item 1).
 *   R3 desiredRowSize is real-valued (Appendix item 3); a tie in the
 *      |#+|S|-d| >= |#-d| test starts a new row.
 *   R4 GetClumpsPartition gives ONE fresh label to each x-tie run with mixed
 *      Q labels (Appendix item 5 keeps equal x-values in one clump; the
 *      worked example, Fig. getclumps, puts the whole x = 1 run in clump 1).
 *   R5 khat = floor(c * x) with x = floor(B / y), at least 1 (Appendix
 *      item 7 quotes khat = cx); superclumps only when k > khat.
 *   R6 OptimizeXAxis DP: candidate s runs over [l-1, t] (s = t is an empty
 *      last column); the first maximum in increasing s wins.
 *   R7 columns beyond the number k of superclumps add nothing:
 *      I(l) = I(k) for l > k, and I = 0 when k = 1.
 *   R8 each orientation is normalised by log min(l, yhat) with its own yhat
 *      (Appendix item 4); min(l, yhat) < 2 gives 0.
 *   R9 MCN uses log2 and epsilon = 0 over x*y <= B (Appendix item 2).
 *   R10 a sample whose x or y is not finite is dropped from that pair.
 *   R11 Pearson rho (reported beside the MINE statistics, Fig. 1) is the
 *      two-pass textbook form over the pair's finite samples, NaN when fewer
 *      than two remain or a variance is zero; the non-linearity index the
 *      paper names without a formula is MIC - rho^2 (the MINE statistics'
 *      original definition), for pairs whose score is valid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_E_PARAM 1
#define ORACLE_E_TOO_FEW 2
#define ORACLE_E_CONSTANT 3
#define ORACLE_E_NOMEM 4

/* ------------------------------------------------------------------------ */
/* Sorting: stable argsort by value (merge sort; ties keep index order).     */
/* ------------------------------------------------------------------------ */

static void merge_pass(const double *v, const int *src, int *dst, int lo,
                       int mid, int hi)
{
    int i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (v[src[j]] < v[src[i]])
            dst[o++] = src[j++];
        else
            dst[o++] = src[i++];
    }
    while (i < mid) dst[o++] = src[i++];
    while (j < hi) dst[o++] = src[j++];
}

/* order[p] = index of the sample at sorted position p. */
static int argsort(const double *v, int n, int *order)
{
    int *tmp = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!tmp) return ORACLE_E_NOMEM;
    for (int i = 0; i < n; i++) order[i] = i;
    int *a = order, *b = tmp;
    for (int width = 1; width < n; width *= 2) {
        for (int lo = 0; lo < n; lo += 2 * width) {
            int mid = lo + width < n ? lo + width : n;
            int hi = lo + 2 * width < n ? lo + 2 * width : n;
            merge_pass(v, a, b, lo, mid, hi);
        }
        int *t = a; a = b; b = t;
    }
    if (a != order) memcpy(order, a, sizeof(int) * (size_t)n);
    free(tmp);
    return ORACLE_OK;
}

int oracle_argsort(const double *v, int n, int *order)
{
    return argsort(v, n, order);
}

/* ------------------------------------------------------------------------ */
/* B = n^alpha  (Sec. 2C: B(n) = n^alpha; reading R1)                       */
/* ------------------------------------------------------------------------ */

int oracle_B(int n, double alpha)
{
    return (int)floor(pow((double)n, alpha));
}

/* ------------------------------------------------------------------------ */
/* EquipartitionYAxis (SOM Algorithm 3; Appendix items 3 and 4).             */
/*                                                                           */
/* Walk the points in increasing order of v, one tie group S at a time.      */
/* '#' is the number of points already given the current row.  Before S is   */
/* assigned, a new row starts if # != 0 and |# + |S| - d| >= |# - d|, where  */
/* d (desiredRowSize) is n/y for the first row and (n - i + 1)/(y - r + 1)   */
/* afterwards, i being the 1-based sorted index of S's first point and r the */
/* 1-based new row.  d is a real number (reading R3).                        */
/* Q[i] receives the 0-based row of sample i; the return value is yhat, the  */
/* number of rows used.                                                      */
/* ------------------------------------------------------------------------ */

int oracle_equipartition(const double *v, int n, int y, int *Q)
{
    if (n <= 0 || y < 1) return 0;
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    if (!order) return -ORACLE_E_NOMEM;
    argsort(v, n, order);

    int curr_row = 1;           /* 1-based, as in the algorithm */
    double desired = (double)n / (double)y;
    int count = 0;              /* '#': points in the current row */
    int i = 0;                  /* 0-based sorted index of S's first point */
    while (i < n) {
        int j = i + 1;
        while (j < n && v[order[j]] == v[order[i]]) j++;
        int s = j - i;          /* |S| */
        if (count != 0 &&
            fabs((double)count + (double)s - desired) >= fabs((double)count - desired)) {
            curr_row += 1;
            /* (n - i + 1) / (y - currRow + 1) with a 1-based i = this i + 1 */
            desired = (double)(n - i) / (double)(y - curr_row + 1);
            count = 0;
        }
        for (int p = i; p < j; p++) Q[order[p]] = curr_row - 1;
        count += s;
        i = j;
    }
    free(order);
    return curr_row;
}

/* ------------------------------------------------------------------------ */
/* GetClumpsPartition (Appendix item 5; worked example Fig. getclumps).     */
/*                                                                           */
/* Definition used here: walk the points in increasing u.  A tie run (the    */
/* maximal set of consecutive points sharing one u-value) must stay inside   */
/* one clump.  A run whose points all lie in the same row keeps that row as  */
/* its label; a run spread over several rows gets a label of its own that    */
/* no other run and no row shares (reading R4: one label for the whole run). */
/* Clumps are then the maximal stretches of consecutive points with equal    */
/* labels.  P[i] receives the 0-based clump of sample i (clumps numbered in  */
/* increasing u); the return value is the number k of clumps.                */
/* ------------------------------------------------------------------------ */

int oracle_clumps(const double *u, const int *Q, int n, int *P)
{
    if (n <= 0) return 0;
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    long *label = (long *)malloc(sizeof(long) * (size_t)n);
    if (!order || !label) { free(order); free(label); return -ORACLE_E_NOMEM; }
    argsort(u, n, order);

    /* label of every sorted position, one tie run at a time */
    long runs = 0;
    int a = 0;
    while (a < n) {
        int b = a + 1;
        while (b < n && u[order[b]] == u[order[a]]) b++;
        int one_row = 1;
        for (int p = a + 1; p < b; p++)
            if (Q[order[p]] != Q[order[a]]) one_row = 0;
        runs += 1;
        /* rows are >= 0, so a negative run number never equals a row */
        long lab = one_row ? (long)Q[order[a]] : -runs;
        for (int p = a; p < b; p++) label[p] = lab;
        a = b;
    }

    /* a new clump wherever the label changes */
    int clump = 0;
    for (int p = 0; p < n; p++) {
        if (p > 0 && label[p] != label[p - 1]) clump += 1;
        P[order[p]] = clump;
    }
    free(order);
    free(label);
    return clump + 1;
}

/* ------------------------------------------------------------------------ */
/* GetSuperclumpsPartition (Appendix items 6-7, Algorithm                    */
/* GetSuperclumpsPartition).                                                 */
/*                                                                           */
/* Clumps first; if there are more than khat of them, EquipartitionYAxis is  */
/* run on the auxiliary set whose second coordinate is the clump label, with */
/* khat as the number of rows, and the result is the superclump map.        */
/* P[i] receives the 0-based superclump of sample i; returns their number.   */
/* ------------------------------------------------------------------------ */

int oracle_superclumps(const double *u, const int *Q, int n, int khat, int *P)
{
    int k = oracle_clumps(u, Q, n, P);
    if (k < 0) return k;
    if (k > khat) {
        double *lab = (double *)malloc(sizeof(double) * (size_t)n);
        int *Pn = (int *)malloc(sizeof(int) * (size_t)n);
        if (!lab || !Pn) { free(lab); free(Pn); return -ORACLE_E_NOMEM; }
        for (int i = 0; i < n; i++) lab[i] = (double)P[i];
        k = oracle_equipartition(lab, n, khat, Pn);
        memcpy(P, Pn, sizeof(int) * (size_t)n);
        free(lab);
        free(Pn);
    }
    return k;
}

/* khat of reading R5 */
int oracle_khat(int B, int y, double c)
{
    int x = B / y;
    int kh = (int)floor(c * (double)x);
    return kh < 1 ? 1 : kh;
}

/* ------------------------------------------------------------------------ */
/* Entropy terms (Appendix item 10a-b; nats; item 9: double precision).      */
/*   L(m) = m ln m, L(0) = 0.                                                */
/*   H(Q) = ln n - sum_r L(q_r) / n.                                         */
/*   E(s,t) = L(c_t - c_s) - sum_r L(cum[r][t] - cum[r][s])                  */
/*          = (c_t - c_s) * H(Q restricted to the column (c_s, c_t]),        */
/* summed in increasing r.  With this, for a column partition P of the n     */
/* points, I(P;Q) = H(Q) + H(P) - H(P,Q) = H(Q) - sum_columns E / n.         */
/* ------------------------------------------------------------------------ */

static double Lfun(long m)
{
    return m > 0 ? (double)m * log((double)m) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* OptimizeXAxis (SOM Algorithm 2 with the precomputations of Appendix       */
/* item 10).  The objective of its step for (t, l),                          */
/*   F(s,t,l) = H(<c_0..c_s,c_t>) - H(<c_0..c_s,c_t>, Q) on the first c_t    */
/*   points, equals (W(s,l-1) - E(s,t)) / c_t, so the maximising s is the    */
/*   same as that of W(s,l-1) - E(s,t) and the table of optima is            */
/*     W(t,1) = -E(0,t)                                                      */
/*     W(t,l) = max_{s in [l-1, t]} W(s,l-1) - E(s,t),   l <= t <= k         */
/* (reading R6: first maximum in increasing s).  Then                        */
/*     I(l) = H(Q) + W(k,l) / n      for 2 <= l <= min(x, k)                 */
/* and reading R7 beyond k.                                                  */
/*                                                                           */
/* Inputs: u (column variable), Q (0-based rows, yhat of them), x (largest   */
/* column count), khat.  Outputs: I_out[l-2] for l = 2..x; cuts_out, if not  */
/* NULL, the chosen partition of each l as the l-1 column ends (superclump   */
/* indices s_1 <= ... <= s_{l-1}, a repeated index being an empty column),   */
/* packed at offset (l-2)(l-1)/2; -1 where l > k.  k_out gets k; sc_ends, if */
/* not NULL and room for k+1 ints is given by sc_cap, gets c_0..c_k.         */
/* ------------------------------------------------------------------------ */

int oracle_optimize_x_axis(const double *u, const int *Q, int n, int yhat,
                           int x, int khat, double *I_out, int *cuts_out,
                           int *k_out, int *sc_ends, int sc_cap)
{
    int rc = ORACLE_OK;
    int *P = (int *)malloc(sizeof(int) * (size_t)n);
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    if (!P || !order) { free(P); free(order); return ORACLE_E_NOMEM; }
    int k = oracle_superclumps(u, Q, n, khat, P);
    if (k < 0) { free(P); free(order); return ORACLE_E_NOMEM; }
    argsort(u, n, order);
    if (k_out) *k_out = k;

    /* superclump ends c_0 = 0 < c_1 < ... < c_k = n in sorted positions */
    int *cend = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    /* cum[r][t]: points of row r among the first t superclumps */
    long *cum = (long *)calloc((size_t)yhat * (size_t)(k + 1), sizeof(long));
    double *E = (double *)malloc(sizeof(double) * (size_t)(k + 1) * (size_t)(k + 1));
    double *W = (double *)malloc(sizeof(double) * (size_t)(k + 1) * (size_t)(x + 1));
    int *A = (int *)malloc(sizeof(int) * (size_t)(k + 1) * (size_t)(x + 1));
    if (!cend || !cum || !E || !W || !A) { rc = ORACLE_E_NOMEM; goto done; }

    cend[0] = 0;
    for (int p = 0; p < n; p++) {
        int t = P[order[p]];
        cend[t + 1] = p + 1;
    }
    if (sc_ends && sc_cap >= k + 1)
        for (int t = 0; t <= k; t++) sc_ends[t] = cend[t];

    for (int t = 1; t <= k; t++) {
        for (int r = 0; r < yhat; r++) cum[(size_t)r * (k + 1) + t] = cum[(size_t)r * (k + 1) + t - 1];
        for (int p = cend[t - 1]; p < cend[t]; p++)
            cum[(size_t)Q[order[p]] * (k + 1) + t] += 1;
    }

    /* H(Q) from the row totals */
    double sumL = 0.0;
    for (int r = 0; r < yhat; r++) sumL += Lfun(cum[(size_t)r * (k + 1) + k]);
    double HQ = log((double)n) - sumL / (double)n;

    /* entropy matrix E(s,t), s <= t (Appendix item 10b) */
    for (int s = 0; s <= k; s++) {
        for (int t = s; t <= k; t++) {
            double e = Lfun((long)cend[t] - (long)cend[s]);
            for (int r = 0; r < yhat; r++)
                e -= Lfun(cum[(size_t)r * (k + 1) + t] - cum[(size_t)r * (k + 1) + s]);
            E[(size_t)s * (k + 1) + t] = e;
        }
    }
#define EM(s, t) E[(size_t)(s) * (k + 1) + (t)]
#define WM(t, l) W[(size_t)(t) * (x + 1) + (l)]
#define AM(t, l) A[(size_t)(t) * (x + 1) + (l)]

    for (int t = 1; t <= k; t++) { WM(t, 1) = -EM(0, t); AM(t, 1) = 0; }
    int lmax = x < k ? x : k;
    for (int l = 2; l <= lmax; l++) {
        for (int t = l; t <= k; t++) {
            double best = -INFINITY;
            int arg = -1;
            for (int s = l - 1; s <= t; s++) {
                double v = WM(s, l - 1) - EM(s, t);
                if (v > best) { best = v; arg = s; }
            }
            WM(t, l) = best;
            AM(t, l) = arg;
        }
    }

    for (int l = 2; l <= x; l++) {
        double I;
        if (k <= 1)
            I = 0.0;
        else if (l <= k)
            I = HQ + WM(k, l) / (double)n;
        else
            I = HQ + WM(k, k) / (double)n;
        I_out[l - 2] = I;
        if (cuts_out) {
            int *cut = cuts_out + (size_t)(l - 2) * (size_t)(l - 1) / 2;
            if (l <= k) {
                int t = k;
                for (int ll = l; ll >= 2; ll--) {
                    int s = AM(t, ll);
                    cut[ll - 2] = s;
                    t = s;
                }
            } else {
                for (int j = 0; j < l - 1; j++) cut[j] = -1;
            }
        }
    }
#undef EM
#undef WM
#undef AM
done:
    free(P); free(order); free(cend); free(cum); free(E); free(W); free(A);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Characteristic matrix (SOM Algorithm 5; Appendix items 1 and 4).          */
/* For orientation o = 0 the rows equipartition y and the columns optimise   */
/* over x; o = 1 swaps the roles.  For every row count r = 2..floor(B/2):    */
/*   Q = EquipartitionYAxis(row variable, r), x_max = floor(B/r),            */
/*   I(l, r) = OptimizeXAxis(column variable, Q, x_max) for l = 2..x_max,    */
/*   M_o(l, r) = I(l, r) / log min(l, yhat)        (reading R8)              */
/* and M(x, y) = max(M_0(x, y), M_1(y, x)) over x*y <= B (reading R2).       */
/*                                                                           */
/* M is stored per pair as the cells (x, y), x, y >= 2, xy <= B, y-major     */
/* then x.  Returns the status; stats = {MIC, MAS, MEV, MCN}; info =        */
/* {n_used, B, mcn_xy, m_cells, yhat_0_at_2, yhat_1_at_2}.                   */
/* ------------------------------------------------------------------------ */

int oracle_m_cells(int B)
{
    int cells = 0;
    for (int y = 2; y <= B / 2; y++) cells += B / y - 1;
    return cells;
}

/* index of cell (x, y) in the y-major layout */
static int cell_index(int B, int x, int y)
{
    int idx = 0;
    for (int yy = 2; yy < y; yy++) idx += B / yy - 1;
    return idx + (x - 2);
}

int oracle_check_param(double alpha, double c)
{
    /* Sec. C++ example: the MINE constructor rejects invalid parameters;
       the accepted ranges are 0 < alpha <= 1 and c > 0. */
    if (!(alpha > 0.0 && alpha <= 1.0)) return ORACLE_E_PARAM;
    if (!(c > 0.0) || !isfinite(c)) return ORACLE_E_PARAM;
    return ORACLE_OK;
}

/* The characteristic matrix of one pair whose samples are already clean. */
static int score_clean(const double *xv, const double *yv, int n, double alpha,
                       double c, double *M, double *stats, int *info)
{
    int B = oracle_B(n, alpha);
    info[0] = n;
    info[1] = B;
    info[2] = 0;
    info[3] = 0;
    info[4] = 0;
    info[5] = 0;
    stats[0] = stats[1] = stats[2] = stats[3] = 0.0;
    if (n < 4 || B < 4) return ORACLE_E_TOO_FEW;

    int cells = oracle_m_cells(B);
    info[3] = cells;
    double *M0 = (double *)calloc((size_t)cells, sizeof(double));
    double *M1 = (double *)calloc((size_t)cells, sizeof(double));
    double *Ib = (double *)malloc(sizeof(double) * (size_t)(B + 1));
    int *Q = (int *)malloc(sizeof(int) * (size_t)n);
    if (!M0 || !M1 || !Ib || !Q) { free(M0); free(M1); free(Ib); free(Q); return ORACLE_E_NOMEM; }

    int status = ORACLE_OK;
    for (int o = 0; o < 2; o++) {
        const double *colv = o == 0 ? xv : yv;   /* optimised axis */
        const double *rowv = o == 0 ? yv : xv;   /* equipartitioned axis */
        double *Mo = o == 0 ? M0 : M1;
        for (int r = 2; r <= B / 2; r++) {
            int yhat = oracle_equipartition(rowv, n, r, Q);
            if (r == 2) info[4 + o] = yhat;
            if (yhat < 2) status = ORACLE_E_CONSTANT;
            int xmax = B / r;
            int khat = oracle_khat(B, r, c);
            int k;
            int rc = oracle_optimize_x_axis(colv, Q, n, yhat, xmax, khat, Ib, NULL, &k, NULL, 0);
            if (rc != ORACLE_OK) { status = rc; goto out; }
            for (int l = 2; l <= xmax; l++) {
                int mn = l < yhat ? l : yhat;
                double val = mn < 2 ? 0.0 : Ib[l - 2] / log((double)mn);
                /* o = 0: l columns on x, r rows on y  -> cell (l, r)
                   o = 1: l columns on y, r rows on x  -> M_1(l, r) */
                Mo[cell_index(B, l, r)] = val;
            }
        }
    }

    /* combine the two orientations: M(x,y) = max(M_0(x,y), M_1(y,x)) */
    for (int y = 2; y <= B / 2; y++)
        for (int x = 2; x <= B / y; x++) {
            double a = M0[cell_index(B, x, y)];
            double b = M1[cell_index(B, y, x)];
            M[cell_index(B, x, y)] = a > b ? a : b;
        }

    /* statistics (Sec. 1 and Appendix items 1-2) */
    double mic = -INFINITY, mas = 0.0, mev = -INFINITY;
    for (int y = 2; y <= B / 2; y++)
        for (int x = 2; x <= B / y; x++) {
            double m = M[cell_index(B, x, y)];
            if (m > mic) mic = m;
            double d = fabs(m - M[cell_index(B, y, x)]);
            if (d > mas) mas = d;
            if ((x == 2 || y == 2) && m > mev) mev = m;
        }
    long mcn_xy = -1;
    for (int y = 2; y <= B / 2; y++)
        for (int x = 2; x <= B / y; x++) {
            double m = M[cell_index(B, x, y)];
            if (m >= mic && (mcn_xy < 0 || (long)x * y < mcn_xy)) mcn_xy = (long)x * y;
        }
    stats[0] = mic;
    stats[1] = mas;
    stats[2] = mev;
    stats[3] = log2((double)mcn_xy);
    info[2] = (int)mcn_xy;
out:
    free(M0); free(M1); free(Ib); free(Q);
    return status;
}

/* Drop the samples where x or y is not finite (reading R10) and score. */
int oracle_score_pair(const double *x, const double *y, int n, double alpha,
                      double c, double *M, double *stats, int *info)
{
    info[0] = info[1] = info[2] = info[3] = info[4] = info[5] = 0;
    stats[0] = stats[1] = stats[2] = stats[3] = 0.0;
    int rc = oracle_check_param(alpha, c);
    if (rc != ORACLE_OK) return rc;
    double *xc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *yc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!xc || !yc) { free(xc); free(yc); return ORACLE_E_NOMEM; }
    int m = 0;
    for (int i = 0; i < n; i++) {
        if (isfinite(x[i]) && isfinite(y[i])) {
            xc[m] = x[i];
            yc[m] = y[i];
            m++;
        }
    }
    rc = score_clean(xc, yc, m, alpha, c, M, stats, info);
    free(xc);
    free(yc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A batch of pairs of variables: vars is [p][n] row-major (one variable per */
/* row, as in the paper's variables-by-samples files); pairs is [npairs][2]. */
/* Pair i uses alphas[i] when alphas is not NULL, else alpha (B = n^alpha is */
/* a per-pair quantity, Sec. 2C).  M_offsets[i] is where pair i's cells     */
/* start in M (or M is NULL).  stats is [npairs][4], info [npairs][6],      */
/* status [npairs].  Pairs are independent and are spread over nthreads     */
/* OpenMP threads.                                                          */
/* ------------------------------------------------------------------------ */

static void score_one(const double *vars, int n, const int *pairs, long i, double alpha,
                      double c, double *stats, int *info, int *status, double *M,
                      const long *M_offsets, double **Mbuf, int *cap)
{
    const double *xv = vars + (size_t)pairs[2 * i] * (size_t)n;
    const double *yv = vars + (size_t)pairs[2 * i + 1] * (size_t)n;
    int need = oracle_m_cells(oracle_B(n, alpha));
    if (need > *cap) {
        free(*Mbuf);
        *cap = need;
        *Mbuf = (double *)malloc(sizeof(double) * (size_t)*cap);
    }
    status[i] = oracle_score_pair(xv, yv, n, alpha, c, *Mbuf, stats + 4 * i, info + 6 * i);
    if (M && M_offsets)
        memcpy(M + M_offsets[i], *Mbuf, sizeof(double) * (size_t)info[6 * i + 3]);
}

static int score_batch(const double *vars, int n, const int *pairs, long npairs,
                       double alpha, const double *alphas, double c, double *stats,
                       int *info, int *status, double *M, const long *M_offsets,
                       int nthreads)
{
    for (long i = 0; i < npairs; i++) {
        int rc = oracle_check_param(alphas ? alphas[i] : alpha, c);
        if (rc != ORACLE_OK) return rc;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
        int cap = 1 << 12;
        double *Mbuf = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
        for (long i = 0; i < npairs; i++)
            score_one(vars, n, pairs, i, alphas ? alphas[i] : alpha, c, stats, info, status, M,
                      M_offsets, &Mbuf, &cap);
        free(Mbuf);
    }
#else
    (void)nthreads;
    int cap = 1 << 12;
    double *Mbuf = (double *)malloc(sizeof(double) * (size_t)cap);
    for (long i = 0; i < npairs; i++)
        score_one(vars, n, pairs, i, alphas ? alphas[i] : alpha, c, stats, info, status, M,
                  M_offsets, &Mbuf, &cap);
    free(Mbuf);
#endif
    return ORACLE_OK;
}

int oracle_score_batch(const double *vars, int p, int n, const int *pairs,
                       long npairs, double alpha, double c, double *stats,
                       int *info, int *status, double *M, const long *M_offsets,
                       int nthreads)
{
    (void)p;
    int rc = oracle_check_param(alpha, c);
    if (rc != ORACLE_OK) return rc;
    return score_batch(vars, n, pairs, npairs, alpha, NULL, c, stats, info, status, M,
                       M_offsets, nthreads);
}

int oracle_score_batch_alphas(const double *vars, int p, int n, const int *pairs,
                              long npairs, const double *alphas, double c, double *stats,
                              int *info, int *status, double *M, const long *M_offsets,
                              int nthreads)
{
    (void)p;
    return score_batch(vars, n, pairs, npairs, 0.0, alphas, c, stats, info, status, M,
                       M_offsets, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Pearson correlation, the linear statistic the paper reports beside the    */
/* four MINE statistics (Fig. 1 caption; SI Sec. 2A: "four MINE statistics,  */
/* Pearson and non-linearity"), over the samples where x and y are both      */
/* finite (reading R10).  The textbook two-pass definition: means first,     */
/*   rho = S_xy / sqrt(S_xx * S_yy),  S_ab = sum_i (a_i - mean a)(b_i - mean b) */
/* with every sum in increasing i.  NaN when fewer than two samples remain   */
/* or a variance is zero (reading R11).  *n_used gets the sample count.      */
/* ------------------------------------------------------------------------ */

double oracle_pearson(const double *x, const double *y, int n, int *n_used)
{
    int m = 0;
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < n; i++) {
        if (isfinite(x[i]) && isfinite(y[i])) {
            sx += x[i];
            sy += y[i];
            m++;
        }
    }
    if (n_used) *n_used = m;
    if (m < 2) return NAN;
    const double mx = sx / (double)m, my = sy / (double)m;
    double sxy = 0.0, sxx = 0.0, syy = 0.0;
    for (int i = 0; i < n; i++) {
        if (isfinite(x[i]) && isfinite(y[i])) {
            const double dx = x[i] - mx, dy = y[i] - my;
            sxy += dx * dy;
            sxx += dx * dx;
            syy += dy * dy;
        }
    }
    if (!(sxx > 0.0) || !(syy > 0.0)) return NAN;
    return sxy / sqrt(sxx * syy);
}

/* Threads OpenMP would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
