"""gmine_compute_batch_uneven: pairs of uneven size, each with its own alpha
(B = n^alpha per pair, Sec. 2C), against the oracle, both precisions.

* uneven pairs with missing samples (n log-uniform in [50, 3000], alpha drawn
  from {0.55, 0.6, 0.75}): the plain FP64 path to 1e-9 with exact MCN cells,
  the FP32 path to 1e-4; the plain path's scores and M equal, bit for bit,
  those of gmine_compute_batch on the same pairs with their alpha;
* pair indices outside [0, p) and pairs with fewer than four samples keep
  their statuses, and every other pair is unaffected by them;
* 33,000 small pairs (more than one chunk of 32,768): every pair against the
  oracle, so that the planned order and the chunk boundaries are covered.
"""
import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import gmine, workloads

from gpu_util import compare_pairs

pytestmark = pytest.mark.gpu


def run_uneven(V, P, alphas, precision, want_M=True):
    import torch
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    Pd = torch.from_numpy(np.ascontiguousarray(P, dtype=np.int32)).cuda()
    vals, _ = gmine.alpha_table(alphas)
    ws = gmine.UnevenWorkspace(V.shape[0], V.shape[1], P.shape[0], vals, 15.0, precision)
    scores, M = gmine.compute_batch_uneven(Vd, Pd, alphas, 15.0, precision, want_M=want_M, workspace=ws)
    torch.cuda.synchronize()
    return {"scores": gmine.scores_to_numpy(scores), "M": M.cpu().numpy() if M is not None else None,
            "cells": ws.cells}


@pytest.fixture(scope="module")
def uneven_case():
    V, P, alphas, ns = workloads.config4(n_pairs=48, n_lo=50, n_hi=3000, seed_salt=48)
    ref = oracle.score_batch(V, P, alphas, 15.0, nthreads=0, want_M=True)
    return V, P, alphas, ref


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_uneven_pairs_per_pair_alpha(uneven_case, precision):
    V, P, alphas, ref = uneven_case
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    run = run_uneven(V, P, alphas, precision)
    s = run["scores"]
    assert np.array_equal(s["B"], ref["info"][:, 1])
    errs = compare_pairs(V, P, run, alphas, 15.0, tol, ref=ref)
    print("uneven, per-pair alpha, precision %d: %s" % (precision, errs))


def test_uneven_plain_equals_regular_path_bitwise(uneven_case):
    import torch
    V, P, alphas, _ = uneven_case
    run = run_uneven(V, P, alphas, gmine.PLAIN_FP64)
    Vd = torch.from_numpy(V).cuda()
    for a in np.unique(alphas):
        sel = np.flatnonzero(alphas == a)
        Pd = torch.from_numpy(np.ascontiguousarray(P[sel])).cuda()
        sc, M = gmine.compute_batch(Vd, Pd, float(a), 15.0, gmine.PLAIN_FP64, want_M=True)
        torch.cuda.synchronize()
        reg = gmine.scores_to_numpy(sc)
        cells_reg = gmine.plan(V.shape[0], V.shape[1], len(sel), float(a), 15.0)[0]
        Mr = M.cpu().numpy()
        for j, i in enumerate(sel):
            got = run["scores"][i]
            for key in ("mic", "mas", "mev", "mcn", "n_used", "B", "m_cells", "mcn_xy", "status",
                        "yhat_x", "yhat_y"):
                assert got[key] == reg[j][key], (i, key)
            mc = int(got["m_cells"])
            assert np.array_equal(run["M"][i * run["cells"]:i * run["cells"] + mc],
                                  Mr[j * cells_reg:j * cells_reg + mc]), i


def test_uneven_bad_indices_and_short_pairs():
    V, P, alphas, _ = workloads.config4(n_pairs=6, n_lo=200, n_hi=800, seed_salt=6)
    V = V.copy()
    V[2, 3:] = np.nan                       # pair 1 keeps 3 samples
    P = P.copy()
    P[3, 1] = V.shape[0] + 5                # pair 3 names a variable outside [0, p)
    P[4, 0] = -1
    run = run_uneven(V, P, alphas, gmine.PLAIN_FP64)
    s = run["scores"]
    assert s["status"][1] == gmine.E_TOO_FEW
    assert s["status"][3] == gmine.E_ARG and s["status"][4] == gmine.E_ARG
    ok = np.array([0, 2, 5])
    ref = oracle.score_batch(V, P[ok], alphas[ok], 15.0, nthreads=0)
    got = np.stack([s["mic"][ok], s["mas"][ok], s["mev"][ok], s["mcn"][ok]], axis=1)
    assert np.max(np.abs(got - ref["stats"])) <= 1e-9


def test_uneven_more_pairs_than_one_chunk():
    n_pairs = 33000
    V, P, alphas, ns = workloads.config4(n_pairs=n_pairs, n_lo=20, n_hi=200, seed_salt=33)
    run = run_uneven(V, P, alphas, gmine.PLAIN_FP64, want_M=False)
    ref = oracle.score_batch(V, P, alphas, 15.0, nthreads=0)
    s = run["scores"]
    assert np.array_equal(s["status"], ref["status"])
    assert np.array_equal(s["n_used"], ref["info"][:, 0]) and np.array_equal(s["B"], ref["info"][:, 1])
    ok = ref["status"] != gmine.E_TOO_FEW
    got = np.stack([s["mic"], s["mas"], s["mev"], s["mcn"]], axis=1)
    assert np.max(np.abs(got[ok] - ref["stats"][ok])) <= 1e-9
    assert np.array_equal(s["mcn_xy"][ok], ref["info"][ok, 2])
