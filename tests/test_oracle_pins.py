"""Pins of the FP64 oracle to facts other than itself (no GPU needed).

* the paper's worked example of EquipartitionYAxis + GetClumpsPartition
  (Appendix, Fig. getclumps), exact;
* the paper's C++ example (Sec. Examples), all four printed statistics;
* a closed form of EquipartitionYAxis for distinct values;
* brute force on tiny inputs: the OptimizeXAxis DP against exhaustive search
  over superclump cut subsets, and against exhaustive search over every
  x-partition that respects x-ties (the clump lemma); the whole method
  against exhaustive search over every grid;
* invariants: MIC = 1 for noiseless functional pairs, 0 <= M <= 1, bitwise
  invariance under order-preserving transforms and sample permutations,
  transposition of M when x and y swap;
* Pearson rho: a hand-computed example, exact linear relations, symmetry and
  affine invariance, numpy's corrcoef, missing samples; the non-linearity
  index on a symmetric parabola and a line.

Mutual information in the brute-force checks is the textbook
sum_jr p_jr ln(p_jr / (p_j p_r)), not the oracle's H(Q) - sum E / n form.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def textbook_mi(cols, rows):
    cols = np.asarray(cols)
    rows = np.asarray(rows)
    n = len(cols)
    mi = 0.0
    for j in np.unique(cols):
        pj = np.count_nonzero(cols == j) / n
        for r in np.unique(rows):
            pr = np.count_nonzero(rows == r) / n
            pjr = np.count_nonzero((cols == j) & (rows == r)) / n
            if pjr > 0:
                mi += pjr * math.log(pjr / (pj * pr))
    return mi


def read_kv(path):
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


# ---------------------------------------------------------------- printed pins

def test_worked_example_getclumps():
    rows = np.loadtxt(os.path.join(GOLD, "getclumps_example.txt"))
    a, b, Qp, Pp = rows[:, 0], rows[:, 1], rows[:, 2].astype(int), rows[:, 3].astype(int)
    Q, yhat = oracle.equipartition(b, 3)
    assert yhat == 3
    assert (Q + 1).tolist() == Qp.tolist()
    P, k = oracle.clumps(a, Q)
    assert k == 5
    assert (P + 1).tolist() == Pp.tolist()
    # With khat >= 5 the superclump step keeps the clumps as they are.
    P2, k2 = oracle.superclumps(a, Q, 5)
    assert k2 == 5 and P2.tolist() == P.tolist()


def test_cpp_example_statistics():
    g = read_kv(os.path.join(GOLD, "cpp_example.txt"))
    n = int(g["n"])
    x = np.arange(n, dtype=np.float64) / float(n - 1)
    y = np.sin(10.0 * g["pi"] * x) + x
    r = oracle.score_pair(x, y, g["alpha"], g["c"])
    assert r["status"] == 0
    assert r["B"] == 63
    # six significant digits as printed: half a unit of the last digit
    assert abs(r["mic"] - g["MIC"]) <= 5e-7
    assert abs(r["mas"] - g["MAS"]) <= 5e-7
    assert abs(r["mev"] - g["MEV"]) <= 5e-7
    assert abs(r["mcn"] - g["MCN"]) <= 5e-7
    assert r["mcn_xy"] == 24


# ---------------------------------------------------------- equipartition

def _sizes_from_Q(Q, yhat):
    return [int(np.count_nonzero(Q == r)) for r in range(yhat)]


@pytest.mark.parametrize("n,y", [(14, 3), (300, 2), (301, 2), (1001, 2), (100, 7),
                                 (1340, 37), (50, 25), (13, 5), (7, 7)])
def test_equipartition_distinct_closed_form(n, y):
    """Distinct values: the greedy rule closes a row once its count a reaches
    d - 1/2, d = remaining points / remaining rows, so the row sizes are
    ceil(d - 1/2) in turn and the last row takes the rest."""
    rng = np.random.default_rng(n * 100 + y)
    v = rng.permutation(n).astype(np.float64) + 0.5
    Q, yhat = oracle.equipartition(v, y)
    expect = []
    remaining = n
    for r in range(y):
        if r == y - 1:
            expect.append(remaining)
            break
        d_num, d_den = remaining, y - r          # d = d_num / d_den
        size = -((-(2 * d_num - d_den)) // (2 * d_den))   # ceil(d - 1/2)
        expect.append(size)
        remaining -= size
    expect = [s for s in expect if s > 0]
    assert yhat == len(expect)
    assert _sizes_from_Q(Q, yhat) == expect
    # rows follow the order of v
    order = np.argsort(v, kind="stable")
    assert np.all(np.diff(Q[order]) >= 0)


def test_equipartition_ties_properties():
    rng = np.random.default_rng(7)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        levels = int(rng.integers(1, 12))
        v = rng.integers(0, levels, n).astype(np.float64)
        y = int(rng.integers(1, 10))
        Q, yhat = oracle.equipartition(v, y)
        assert 1 <= yhat <= y
        assert set(Q.tolist()) == set(range(yhat))           # no empty row
        for val in np.unique(v):                               # ties stay together
            assert len(set(Q[v == val].tolist())) == 1
        order = np.argsort(v, kind="stable")
        assert np.all(np.diff(Q[order]) >= 0)                  # rows are intervals
        if len(np.unique(v)) == 1:
            assert yhat == 1
        elif y >= 2:
            assert yhat >= 2


# --------------------------------------------------------------- clumps

def test_clumps_definition_random():
    """Clumps: the maximal runs (in x order) of points with one Q label, except
    that an x-tie run with mixed labels is one clump of its own."""
    rng = np.random.default_rng(11)
    for trial in range(300):
        n = int(rng.integers(1, 40))
        u = rng.integers(0, int(rng.integers(1, 15)), n).astype(np.float64)
        Q = rng.integers(0, int(rng.integers(1, 4)), n).astype(np.int32)
        P, k = oracle.clumps(u, Q)
        order = np.argsort(u, kind="stable")
        us, qs, ps = u[order], Q[order], P[order]
        # independent construction from the definition
        labels = []
        i = 0
        fresh = 0
        while i < n:
            j = i
            while j < n and us[j] == us[i]:
                j += 1
            run = qs[i:j]
            if len(set(run.tolist())) > 1:
                fresh += 1
                labels += [("mixed", fresh)] * (j - i)
            else:
                labels += [("q", int(run[0]))] * (j - i)
            i = j
        expect = [0]
        for m in range(1, n):
            expect.append(expect[-1] + (labels[m] != labels[m - 1]))
        assert ps.tolist() == expect
        assert k == (expect[-1] + 1 if n else 0)


def test_superclumps_distinct_closed_form():
    """Alternating rows on distinct x make every point a clump; merging n
    single-point clumps into khat superclumps is EquipartitionYAxis of n
    distinct values, whose sizes have the closed form above."""
    for n, khat in [(40, 7), (41, 3), (100, 30), (12, 12), (13, 12)]:
        u = np.arange(n, dtype=np.float64)
        Q = (np.arange(n) % 2).astype(np.int32)
        P, k = oracle.superclumps(u, Q, khat)
        sizes = [int(np.count_nonzero(P == t)) for t in range(k)]
        expect = []
        remaining = n
        for r in range(khat):
            if r == khat - 1:
                expect.append(remaining)
                break
            size = -((-(2 * remaining - (khat - r))) // (2 * (khat - r)))
            expect.append(size)
            remaining -= size
        expect = [s for s in expect if s > 0]
        if n <= khat:
            expect = [1] * n
        assert sizes == expect
        assert np.all(np.diff(P) >= 0)


def test_superclumps_merge_whole_clumps():
    rng = np.random.default_rng(5)
    for trial in range(100):
        n = int(rng.integers(5, 80))
        u = rng.integers(0, 30, n).astype(np.float64)
        Q = rng.integers(0, 3, n).astype(np.int32)
        P0, k0 = oracle.clumps(u, Q)
        khat = int(rng.integers(1, 12))
        P, k = oracle.superclumps(u, Q, khat)
        assert k <= max(khat, 1) or k == k0 <= khat
        assert k == min(k, k0)
        # every clump lies in exactly one superclump
        for cl in range(k0):
            assert len(set(P[P0 == cl].tolist())) == 1
        if k0 <= khat:
            assert P.tolist() == P0.tolist()


# ------------------------------------------------------------- DP brute force

def _u_sorted_rows(u, Q):
    order = oracle.argsort(u)
    return order, np.asarray(Q)[order]


@pytest.mark.parametrize("seed", range(40))
def test_dp_matches_exhaustive_cut_subsets(seed):
    """For fixed Q and fixed superclumps, I(l) is the maximum over every way of
    cutting the superclump sequence into at most l columns."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 13))
    u = rng.integers(0, int(rng.integers(3, 14)), n).astype(np.float64)
    v = rng.normal(size=n)
    y = int(rng.integers(2, 5))
    Q, yhat = oracle.equipartition(v, y)
    x = int(rng.integers(2, 7))
    khat = int(rng.integers(1, 9))
    res = oracle.optimize_x_axis(u, Q, yhat, x, khat)
    k = res["k"]
    ends = res["sc_ends"]
    order, qs = _u_sorted_rows(u, Q)
    for l in range(2, x + 1):
        best = -1.0
        for m in range(0, min(l - 1, k - 1) + 1):
            for cut in itertools.combinations(range(1, k), m):
                bounds = [0] + [int(ends[c]) for c in cut] + [n]
                cols = np.zeros(n, dtype=int)
                for j in range(len(bounds) - 1):
                    cols[bounds[j]:bounds[j + 1]] = j
                best = max(best, textbook_mi(cols, qs))
        if k <= 1:
            best = 0.0
        assert abs(res["I"][l - 2] - best) <= 1e-12, (l, res["I"][l - 2], best)
        # the reported partition attains I(l)
        if l <= k:
            cut = res["cuts"][l - 2]
            assert cut == sorted(cut) and cut[-1] <= k
            bounds = [0] + [int(ends[c]) for c in cut] + [n]
            cols = np.zeros(n, dtype=int)
            for j in range(len(bounds) - 1):
                cols[bounds[j]:bounds[j + 1]] = j
            assert abs(textbook_mi(cols, qs) - res["I"][l - 2]) <= 1e-12


@pytest.mark.parametrize("seed", range(25))
def test_dp_clump_lemma_exhaustive_over_x_partitions(seed):
    """With khat above the clump count (no superclumps), I(l) equals the best
    mutual information over EVERY partition of the x-axis into at most l
    columns that keeps x-ties together: cutting inside a clump never helps."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(4, 12))
    u = rng.integers(0, int(rng.integers(3, 12)), n).astype(np.float64)
    v = rng.integers(0, 5, n).astype(np.float64)
    y = int(rng.integers(2, 4))
    Q, yhat = oracle.equipartition(v, y)
    x = int(rng.integers(2, 6))
    res = oracle.optimize_x_axis(u, Q, yhat, x, 10 ** 6)
    order, qs = _u_sorted_rows(u, Q)
    us = u[order]
    cut_pos = [m for m in range(1, n) if us[m] != us[m - 1]]
    for l in range(2, x + 1):
        best = 0.0
        for m in range(0, min(l - 1, len(cut_pos)) + 1):
            for cut in itertools.combinations(cut_pos, m):
                bounds = [0] + list(cut) + [n]
                cols = np.zeros(n, dtype=int)
                for j in range(len(bounds) - 1):
                    cols[bounds[j]:bounds[j + 1]] = j
                best = max(best, textbook_mi(cols, qs))
        assert abs(res["I"][l - 2] - best) <= 1e-12, (l, res["I"][l - 2], best)


def _best_grid_mi(u, v, nx, ny):
    """Exhaustive max MI over every grid with <= nx columns and <= ny rows
    that keeps ties together on both axes."""
    n = len(u)
    ou = np.argsort(u, kind="stable")
    ov = np.argsort(v, kind="stable")
    us, vs = u[ou], v[ov]
    cu = [m for m in range(1, n) if us[m] != us[m - 1]]
    cv = [m for m in range(1, n) if vs[m] != vs[m - 1]]
    best = 0.0
    col_parts = []
    for m in range(0, min(nx - 1, len(cu)) + 1):
        for cut in itertools.combinations(cu, m):
            lab = np.zeros(n, dtype=int)
            b = [0] + list(cut) + [n]
            for j in range(len(b) - 1):
                lab[ou[b[j]:b[j + 1]]] = j
            col_parts.append(lab)
    for m in range(0, min(ny - 1, len(cv)) + 1):
        for cut in itertools.combinations(cv, m):
            rl = np.zeros(n, dtype=int)
            b = [0] + list(cut) + [n]
            for j in range(len(b) - 1):
                rl[ov[b[j]:b[j + 1]]] = j
            for cl in col_parts:
                best = max(best, textbook_mi(cl, rl))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_method_below_exhaustive_grid_optimum(seed):
    """Every I(x, y) the method finds is at most the best over all x-by-y
    grids; M lies in [0, 1]."""
    rng = np.random.default_rng(3000 + seed)
    n = 8
    u = rng.integers(0, 6, n).astype(np.float64)
    v = u + rng.integers(0, 3, n)
    B = oracle.B_of(n, 1.0)
    for y in range(2, B // 2 + 1):
        Q, yhat = oracle.equipartition(v, y)
        xmax = B // y
        res = oracle.optimize_x_axis(u, Q, yhat, xmax, oracle.khat_of(B, y, 15))
        for l in range(2, xmax + 1):
            star = _best_grid_mi(u, v, l, y)
            assert res["I"][l - 2] <= star + 1e-12
    r = oracle.score_pair(u, v, 1.0, 15)
    assert np.all(r["M"] >= -1e-12) and np.all(r["M"] <= 1 + 1e-12)


# --------------------------------------------------------------- invariants

@pytest.mark.parametrize("kind", ["linear", "parabola", "sine"])
def test_mic_one_for_noiseless_functions(kind):
    rng = np.random.default_rng(42)
    n = 300
    x = rng.uniform(0, 1, n)
    y = {"linear": x, "parabola": 4 * x * (1 - x), "sine": np.sin(8 * np.pi * x)}[kind]
    r = oracle.score_pair(x, y, 0.6, 15)
    assert r["status"] == 0 and r["B"] == 30
    assert abs(r["mic"] - 1.0) <= 1e-12


def test_independent_low_and_bounded():
    rng = np.random.default_rng(43)
    x = rng.uniform(0, 1, 300)
    y = rng.uniform(0, 1, 300)
    r = oracle.score_pair(x, y, 0.6, 15)
    assert 0.0 <= r["mic"] < 0.5
    assert np.all(r["M"] >= 0.0) and np.all(r["M"] <= 1.0 + 1e-12)


def test_order_preserving_transform_and_permutation_bitwise():
    rng = np.random.default_rng(44)
    n = 200
    x = rng.normal(size=n)
    y = np.sin(3 * x) + 0.3 * rng.normal(size=n)
    y[::7] = np.round(y[::7], 1)          # some ties
    base = oracle.score_pair(x, y, 0.6, 15)
    # exact order-preserving maps: power-of-two scaling and dense ranks
    ranks = np.unique(y, return_inverse=True)[1].astype(np.float64)
    t = oracle.score_pair(4.0 * x, ranks, 0.6, 15)
    assert np.array_equal(base["M"], t["M"])
    perm = rng.permutation(n)
    pm = oracle.score_pair(x[perm], y[perm], 0.6, 15)
    assert np.array_equal(base["M"], pm["M"])
    for key in ("mic", "mas", "mev", "mcn"):
        assert base[key] == t[key] == pm[key]


def test_swap_transposes_M():
    rng = np.random.default_rng(45)
    n = 250
    x = rng.uniform(size=n)
    y = x ** 2 + 0.2 * rng.normal(size=n)
    a = oracle.score_pair(x, y, 0.6, 15)
    b = oracle.score_pair(y, x, 0.6, 15)
    cells = oracle.cell_layout(a["B"])
    idx = {c: i for i, c in enumerate(cells)}
    for (cx, cy), i in idx.items():
        assert a["M"][i] == b["M"][idx[(cy, cx)]]
    assert a["mic"] == b["mic"] and a["mas"] == b["mas"] and a["mev"] == b["mev"]


def test_large_c_removes_superclumps():
    """Sec. c-sweep (Fig. otucomparison): once khat exceeds every clump count
    the superclump step is idle and the result no longer depends on c."""
    rng = np.random.default_rng(46)
    x = rng.uniform(size=120)
    y = x + 0.5 * rng.normal(size=120)
    a = oracle.score_pair(x, y, 0.6, 120.0)
    b = oracle.score_pair(x, y, 0.6, 1e6)
    assert np.array_equal(a["M"], b["M"])


def test_nan_dropped_and_status():
    rng = np.random.default_rng(47)
    x = rng.uniform(size=100)
    y = x + 0.1 * rng.normal(size=100)
    xn = x.copy()
    xn[[3, 50]] = np.nan
    yn = y.copy()
    yn[7] = np.inf
    keep = np.ones(100, bool)
    keep[[3, 50, 7]] = False
    a = oracle.score_pair(xn, yn, 0.6, 15)
    b = oracle.score_pair(x[keep], y[keep], 0.6, 15)
    assert a["n_used"] == 97
    assert np.array_equal(a["M"], b["M"])
    c = oracle.score_pair(np.ones(50), y[:50], 0.6, 15)
    assert oracle.STATUS[c["status"]] == "E_CONSTANT" and c["mic"] == 0.0
    d = oracle.score_pair(x[:3], y[:3], 0.6, 15)
    assert oracle.STATUS[d["status"]] == "E_TOO_FEW"
    e = oracle.score_pair(x, y, 1.5, 15)
    assert oracle.STATUS[e["status"]] == "E_PARAM"


def test_B_reading():
    assert oracle.B_of(1340, 0.6) == 75
    assert oracle.B_of(300, 0.6) == 30
    assert oracle.B_of(1000, 0.6) == 63
    assert oracle.B_of(100000, 0.6) == 999   # pow() rounds just below 1000
    assert oracle.m_cells(75) == len(oracle.cell_layout(75)) == 189


def test_batch_equals_single():
    V, P = np.random.default_rng(3).normal(size=(6, 120)), np.array([[0, 1], [2, 5], [4, 3]])
    out = oracle.score_batch(V, P, 0.6, 15, nthreads=2, want_M=True)
    for i, (a, b) in enumerate(P):
        r = oracle.score_pair(V[a], V[b], 0.6, 15)
        assert out["stats"][i].tolist() == [r["mic"], r["mas"], r["mev"], r["mcn"]]
        off = out["M_offsets"][i]
        assert np.array_equal(out["M"][off:off + r["m_cells"]], r["M"])


# ------------------------------------------------- readings of silent points

def _three_level_pair(sizes, seed):
    """A noiseless pair built on a variable with three distinct values: V
    takes 0, 1, 2 on groups of the given sizes (shuffled), U = 10 V + 3 (the
    same order, so both variables have the same three tie groups)."""
    rng = np.random.default_rng(seed)
    v = np.repeat(np.arange(3, dtype=np.float64), sizes)
    v = v[rng.permutation(len(v))]
    return 10.0 * v + 3.0, v


def _h(probs):
    return -sum(p * math.log(p) for p in probs if p > 0)


@pytest.mark.parametrize("sizes", [(100, 100, 100), (50, 120, 130), (40, 200, 60)])
def test_normalisation_uses_yhat(sizes):
    """Appendix item 4: I(x, y) is normalised by min(log x, log yhat), yhat
    being the number of rows EquipartitionYAxis actually used.  V takes three
    values on groups of the given sizes and U = 10 V + 3, so both variables
    have the same three tie groups G and every column partition is a function
    of G.  In either orientation (the two are the same here):
      y >= 3 rows: yhat = 3, the rows are G, the clumps are G; I(l) = H(G)
        for l >= 3 and, for l = 2, the better of the two cuts of G;
      y = 2 rows: the greedy rule merges two neighbouring groups (closed form
        below), the clumps are those two rows, so I(l) = H(rows) (reading R7);
    each divided by log min(l, yhat), and M(x, y) the larger of the two
    orientations' (x, y) and (y, x) entries.  Mutual informations are the
    textbook sum, not the oracle's entropy form.  Dividing by log min(x, y)
    instead would lower every cell with x, y >= 4."""
    n = sum(sizes)
    u, v = _three_level_pair(sizes, seed=sum(sizes) + sizes[0])
    for y in range(3, 16):
        Q, yhat = oracle.equipartition(v, y)
        assert yhat == 3
    r = oracle.score_pair(u, v, 0.6, 15)
    B = r["B"]
    assert r["status"] == 0 and B == oracle.B_of(n, 0.6) == 30
    grp = np.round(v).astype(int)
    # 2-row equipartition of three groups: the second group opens row 2 iff
    # |s1 + s2 - n/2| >= |s1 - n/2|, else the third one does
    d = n / 2.0
    rows2 = (grp >= 1) if abs(sizes[0] + sizes[1] - d) >= abs(sizes[0] - d) else (grp >= 2)
    rows2 = rows2.astype(int)
    Q2, yhat2 = oracle.equipartition(v, 2)
    assert yhat2 == 2 and np.array_equal(Q2, rows2)
    h_g = textbook_mi(grp, grp)
    h_cut = max(textbook_mi((grp >= 1).astype(int), grp), textbook_mi((grp >= 2).astype(int), grp))
    h_rows2 = textbook_mi(rows2, rows2)

    def m_o(l, y):
        if y >= 3:
            return (h_g if l >= 3 else h_cut) / math.log(min(l, 3))
        return h_rows2 / math.log(2)

    cells = oracle.cell_layout(B)
    assert (4, 4) in cells and (5, 6) in cells
    want = np.array([max(m_o(x, y), m_o(y, x)) for x, y in cells])
    assert np.max(np.abs(r["M"] - want)) <= 1e-12
    assert abs(r["mic"] - want.max()) <= 1e-12
    assert abs(r["mas"]) <= 1e-12
    mcn = min(x * y for (x, y), m in zip(cells, r["M"]) if m >= r["mic"])
    assert r["mcn_xy"] == mcn


def test_normalisation_yhat_hand_value():
    """A cell computed by hand where yhat < y decides the value: V has three
    values on 4, 4 and 8 of n = 16 points and U = V.  With alpha = 1, B = 16.
    For y = 4 rows the greedy rule keeps one row per group (d = 4: the second
    group opens a row since |4 + 4 - 4| >= |4 - 4|, the third since
    |4 + 8 - 4| >= |4 - 4| with d = 12/3), so yhat = 3; the three clumps give
    I(4, 4) = H(1/4, 1/4, 1/2) = 1.5 ln 2 and M(4, 4) = 1.5 ln 2 / ln 3 =
    0.9464..., where log min(4, 4) would give 0.75."""
    v = np.array([0.0] * 4 + [1.0] * 4 + [2.0] * 8)
    Q, yhat = oracle.equipartition(v, 4)
    assert yhat == 3
    r = oracle.score_pair(v.copy(), v, 1.0, 15)
    assert r["B"] == 16
    idx = {c: i for i, c in enumerate(oracle.cell_layout(16))}
    assert abs(r["M"][idx[(4, 4)]] - 1.5 * math.log(2) / math.log(3)) <= 1e-12
    assert abs(r["M"][idx[(3, 4)]] - 1.5 * math.log(2) / math.log(3)) <= 1e-12


def test_khat_bound_is_cx():
    """Appendix item 7: the superclump count stops at khat = c*x (MINE.jar's
    c*x + 1 is the defect the paper reports).  Alternating rows on distinct x
    give n single-point clumps, so the bound is reached exactly."""
    n = 400
    u = np.arange(n, dtype=np.float64)
    v = np.where(np.arange(n) % 2 == 0, 0.0, 1.0)
    B = oracle.B_of(n, 0.6)          # 36
    for y, c in [(2, 5.0), (3, 2.0), (4, 7.0), (2, 1.0)]:
        Q, yhat = oracle.equipartition(v, y)
        x = B // y
        res = oracle.optimize_x_axis(u, Q, yhat, x, oracle.khat_of(B, y, c))
        assert res["k"] == int(c) * x


def test_dp_first_maximum_wins():
    """Reading R6: among equal candidates the lowest s wins.  Rows 0,1,0,1 on
    four distinct x: cutting after the first or after the third point gives
    the same entropy sum, evaluated to the same double."""
    u = np.arange(4, dtype=np.float64)
    Q = np.array([0, 1, 0, 1], dtype=np.int32)
    res = oracle.optimize_x_axis(u, Q, 2, 2, 1000)
    assert res["k"] == 4
    assert res["cuts"][0] == [1]


def test_dp_empty_column_candidate_is_kept():
    """Reading R6: s runs up to t, so an empty last column (s = t) is a
    candidate and can win when rounding puts every split a hair lower.  On
    this input the l = 5 optimum carries a repeated cut (an empty column) and
    still attains I(5)."""
    u = np.array([14.0, 16.0, 23.0, 0.0, 21.0, 14.0, 16.0, 13.0, 24.0])
    v = np.array([1.0, 2.0, 3.0, 0.0, 2.0, 3.0, 0.0, 0.0, 1.0])
    Q, yhat = oracle.equipartition(v, 2)
    res = oracle.optimize_x_axis(u, Q, yhat, 7, 1000)
    cut = res["cuts"][5 - 2]
    assert len(set(cut)) < len(cut)
    order, qs = _u_sorted_rows(u, Q)
    ends = res["sc_ends"]
    bounds = [0] + [int(ends[c]) for c in cut] + [len(u)]
    cols = np.zeros(len(u), dtype=int)
    for j in range(len(bounds) - 1):
        cols[bounds[j]:bounds[j + 1]] = j
    assert abs(textbook_mi(cols, qs) - res["I"][5 - 2]) <= 1e-12


# ---- Pearson rho (reported beside the MINE statistics, Fig. 1; reading R11)

def test_pearson_hand_example():
    # x = 1..5, y = (2, 4, 5, 4, 5): means 3 and 4, S_xy = 6, S_xx = 10,
    # S_yy = 6, so rho = 6 / sqrt(60) = sqrt(0.6)
    r, m = oracle.pearson([1, 2, 3, 4, 5], [2, 4, 5, 4, 5])
    assert m == 5
    assert abs(r - math.sqrt(0.6)) <= 2e-16


def test_pearson_closed_forms_and_invariants():
    rng = np.random.default_rng(11)
    x = rng.normal(size=400)
    y = 0.3 * x + rng.normal(size=400)
    r, _ = oracle.pearson(x, y)
    # exact linear relations give +-1; rho(x, x) = 1
    assert abs(oracle.pearson(x, 2.5 * x - 7.0)[0] - 1.0) <= 1e-14
    assert abs(oracle.pearson(x, -0.5 * x + 1.0)[0] + 1.0) <= 1e-14
    assert abs(oracle.pearson(x, x)[0] - 1.0) <= 1e-15
    # symmetric; invariant under positive affine maps, sign flips with a
    # negative scale
    assert abs(oracle.pearson(y, x)[0] - r) <= 1e-15
    assert abs(oracle.pearson(3.0 * x + 2.0, 0.25 * y - 9.0)[0] - r) <= 1e-13
    assert abs(oracle.pearson(-x, y)[0] + r) <= 1e-15
    assert -1.0 <= r <= 1.0


def test_pearson_matches_numpy_corrcoef():
    # an independent library routine (numpy's covariance-based corrcoef)
    rng = np.random.default_rng(12)
    for n in (2, 3, 10, 1340):
        x = rng.lognormal(6.0, 1.5, size=n)
        y = np.sin(x / 200.0) + rng.normal(scale=0.3, size=n)
        r, _ = oracle.pearson(x, y)
        assert abs(r - np.corrcoef(x, y)[0, 1]) <= 1e-12


def test_pearson_missing_samples_and_degenerate_cases():
    rng = np.random.default_rng(13)
    x = rng.normal(size=200)
    y = x ** 2 + rng.normal(size=200)
    xm, ym = x.copy(), y.copy()
    xm[::7] = np.nan
    ym[3::11] = np.inf
    keep = np.isfinite(xm) & np.isfinite(ym)
    r, m = oracle.pearson(xm, ym)
    r2, m2 = oracle.pearson(x[keep], y[keep])
    assert m == m2 == int(keep.sum())
    assert r == r2  # the same samples in the same order: the same double
    assert math.isnan(oracle.pearson([1.0], [2.0])[0])               # one sample
    assert math.isnan(oracle.pearson([1.0, 1.0, 1.0], [1.0, 2.0, 3.0])[0])  # zero variance
    assert math.isnan(oracle.pearson([np.nan, 1.0], [1.0, np.nan])[0])      # nothing left


def test_nonlinearity_index():
    # noiseless y = x^2 on a symmetric grid: rho = 0 by symmetry (up to
    # rounding) while MIC is near 1 (a function), so the index is MIC itself
    # and close to 1; a noiseless line has MIC = 1 and rho = 1: index 0
    x = np.linspace(-1.0, 1.0, 201)
    s = oracle.score_pair(x, x * x)
    r, _ = oracle.pearson(x, x * x)
    assert abs(r) <= 1e-13
    idx = oracle.nonlinearity(s["mic"], r)
    assert abs(idx - s["mic"]) <= 1e-25 and idx > 0.99
    s = oracle.score_pair(x, 3.0 * x)
    r, _ = oracle.pearson(x, 3.0 * x)
    assert abs(s["mic"] - 1.0) <= 1e-15
    assert abs(oracle.nonlinearity(s["mic"], r)) <= 1e-14
