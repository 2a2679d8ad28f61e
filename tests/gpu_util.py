"""Helpers of the GPU parity tests: run a batch through the C ABI and compute
the oracle's per-task and per-pair values for the same inputs."""
import numpy as np

import oracle
from paper_1208_4271_gb300 import gmine


def run_batch(V, P, alpha=0.6, c=15.0, precision=gmine.PLAIN_FP64, trace=True, want_M=True):
    import torch
    dev = torch.device("cuda:0")
    Vd = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).to(dev)
    Pd = torch.from_numpy(np.ascontiguousarray(P, dtype=np.int32)).to(dev)
    n = V.shape[1]
    tr, tt = (None, None)
    if trace:
        tr, tt = gmine.alloc_trace(P.shape[0], n, alpha, c)
    scores, M = gmine.compute_batch(Vd, Pd, alpha, c, precision, want_M=want_M, trace=tr)
    torch.cuda.synchronize()
    out = {"scores": gmine.scores_to_numpy(scores),
           "M": M.cpu().numpy() if M is not None else None,
           "cells": gmine.plan(V.shape[0], n, P.shape[0], alpha, c, precision)[0]}
    if trace:
        out["trace"] = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in tt.items()}
    return out


def pair_samples(V, P, i):
    x = V[P[i, 0]]
    y = V[P[i, 1]]
    keep = np.isfinite(x) & np.isfinite(y)
    return x[keep], y[keep]


def oracle_task(V, P, i, o, y, alpha, c):
    """Oracle values of task (pair i, orientation o, row count y)."""
    xs, ys = pair_samples(V, P, i)
    n = len(xs)
    B = oracle.B_of(n, alpha)
    if n < 4 or B < 4 or y > B // 2:
        return None
    U, Vr = (xs, ys) if o == 0 else (ys, xs)
    Q, yhat = oracle.equipartition(Vr, y)
    _, nclumps = oracle.clumps(U, Q)
    x = B // y
    res = oracle.optimize_x_axis(U, Q, yhat, x, oracle.khat_of(B, y, c))
    res.update({"yhat": yhat, "clumps": nclumps, "x": x, "B": B})
    return res


def task_index(i, o, y, n_pairs):
    return ((y - 2) * 2 + o) * n_pairs + i


def compare_tasks(V, P, run, pairs_to_check, alpha, c, check_cuts=True, I_tol=1e-9):
    """Element-by-element comparison of the trace with the oracle.  Returns
    (tasks checked, tasks whose chosen partitions differ)."""
    tr = run["trace"]
    R = tr["R"]
    n_pairs = P.shape[0]
    checked = 0
    differ = 0
    for i in pairs_to_check:
        for o in (0, 1):
            for y in range(2, R + 2):
                t = task_index(i, o, y, n_pairs)
                ref = oracle_task(V, P, i, o, y, alpha, c)
                if ref is None:
                    assert tr["k"][t] == 0, (i, o, y)
                    continue
                k = ref["k"]
                assert tr["yhat"][t] == ref["yhat"], ("yhat", i, o, y)
                assert tr["clumps"][t] == ref["clumps"], ("clumps", i, o, y)
                assert tr["k"][t] == k, ("k", i, o, y, tr["k"][t], k)
                assert np.array_equal(tr["sc_ends"][t, :k + 1], ref["sc_ends"]), ("sc_ends", i, o, y)
                x = ref["x"]
                got_I = tr["I"][t, :x - 1]
                err = np.max(np.abs(got_I - ref["I"])) if x > 1 else 0.0
                assert err <= I_tol, ("I", i, o, y, err)
                cuts_same = True
                for l in range(2, x + 1):
                    off = (l - 2) * (l - 1) // 2
                    got = tr["cuts"][t, off:off + l - 1].tolist()
                    if got != ref["cuts"][l - 2]:
                        cuts_same = False
                if check_cuts:
                    assert cuts_same, ("cuts", i, o, y)
                differ += 0 if cuts_same else 1
                checked += 1
    return checked, differ


def compare_pairs(V, P, run, alpha, c, tol, idx=None, ref=None, check_M=True):
    """Statistics (and M) of the listed pairs against the oracle."""
    if idx is None:
        idx = np.arange(P.shape[0])
    if ref is None:
        ref = oracle.score_batch(V, P[idx], alpha, c, nthreads=0, want_M=check_M)
    s = run["scores"][idx]
    assert np.array_equal(s["status"], ref["status"]), "status"
    assert np.array_equal(s["n_used"], ref["info"][:, 0]), "n_used"
    assert np.array_equal(s["B"], ref["info"][:, 1]), "B"
    got = np.stack([s["mic"], s["mas"], s["mev"], s["mcn"]], axis=1)
    err = np.abs(got - ref["stats"])
    ok = ref["status"] != gmine.E_TOO_FEW
    errs = {"mic": 0.0, "mas": 0.0, "mev": 0.0, "mcn": 0.0}
    if ok.any():
        for j, name in enumerate(("mic", "mas", "mev", "mcn")):
            errs[name] = float(err[ok, j].max())
    if check_M and run["M"] is not None:
        cells = run["cells"]
        mmax = 0.0
        for j, i in enumerate(idx):
            if not ok[j]:
                continue
            mc = int(ref["info"][j, 3])
            a = run["M"][i * cells:i * cells + mc]
            b = ref["M"][ref["M_offsets"][j]:ref["M_offsets"][j] + mc]
            mmax = max(mmax, float(np.max(np.abs(a - b))) if mc else 0.0)
        errs["M"] = mmax
    for name, e in errs.items():
        if name in ("mic", "mas", "mev", "M"):
            assert e <= tol, (name, e, tol)
    if ok.any():
        assert errs["mcn"] <= max(tol, 1e-9) or tol > 1e-9
    if tol <= 1e-9:
        assert np.array_equal(s["mcn_xy"][ok], ref["info"][ok, 2]), "mcn_xy"
    elif check_M and "M" in ref:
        # the float path's MCN (log2 of the smallest xy whose cell equals its
        # MIC exactly) is a step function of near-equal scores; what it must
        # give is a grid whose exact score is within the contract of the
        # exact MIC: some cell with that xy has oracle M >= MIC - 2 tol
        worst = 0.0
        for j, i in enumerate(idx):
            if ref["status"][j] != gmine.OK:
                continue
            B = int(ref["info"][j, 1])
            cells = oracle.cell_layout(B)
            Mref = ref["M"][ref["M_offsets"][j]:ref["M_offsets"][j] + len(cells)]
            xy = int(s["mcn_xy"][j])
            best = max(m for (cx, cy), m in zip(cells, Mref) if cx * cy == xy)
            worst = max(worst, float(ref["stats"][j, 0] - best))
        errs["mcn_cell_gap"] = worst
        assert worst <= 2 * tol, ("mcn cell", worst)
    return errs
