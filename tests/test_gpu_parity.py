"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Plain FP64 path: every integer quantity bit-exact (ranks, Q maps, yhat,
clump counts, superclump ends, chosen partitions) and every score within
1e-9 absolute.  FP32 DP with FP64 re-scoring: MIC, MAS, MEV within 1e-4,
integers of the partition steps still exact, chosen partitions reported.
"""
import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import gmine, workloads

from gpu_util import compare_pairs, compare_tasks, run_batch

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    gmine.lib()


def _dense_rank(v):
    return np.unique(v, return_inverse=True)[1].astype(np.int32)


def test_rank_parity():
    import torch
    V, _ = workloads.config1()
    T, _ = workloads.tie_heavy(p=6, n=333)
    for M in (V, T, np.round(V * 7) / 7):
        perm, rk, groups = gmine.rank(torch.from_numpy(M).cuda())
        torch.cuda.synchronize()
        perm, rk, groups = perm.cpu().numpy(), rk.cpu().numpy(), groups.cpu().numpy()
        for v in range(M.shape[0]):
            assert np.array_equal(perm[v], oracle.argsort(M[v]))
            dr = _dense_rank(M[v])
            assert np.array_equal(rk[v], dr)
            assert groups[v] == dr.max() + 1


@pytest.mark.parametrize("y", [2, 3, 5, 7, 37, 100])
def test_equipartition_parity(y):
    import torch
    V, _ = workloads.config2()
    T, _ = workloads.tie_heavy(p=8, n=500, levels=9)
    for M in (V[:20], T):
        Q, yh = gmine.equipartition(torch.from_numpy(M).cuda(), y)
        torch.cuda.synchronize()
        Q, yh = Q.cpu().numpy(), yh.cpu().numpy()
        for v in range(M.shape[0]):
            q, h = oracle.equipartition(M[v], y)
            assert yh[v] == h
            assert np.array_equal(Q[v], q)


def test_worked_example_on_gpu():
    """The paper's worked example (Fig. getclumps): Q of y = 3 rows."""
    import torch
    b = np.array([1, 2, 3, 4, 3, 4, 5, 6, 6, 6, 5, 3, 2, 1], dtype=np.float64)
    Q, yh = gmine.equipartition(torch.from_numpy(b[None, :]).cuda(), 3)
    torch.cuda.synchronize()
    assert int(yh[0]) == 3
    assert (Q.cpu().numpy()[0] + 1).tolist() == [1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 3, 2, 1, 1]


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_cpp_example_on_gpu(precision):
    V, P = workloads.cpp_example()
    r = gmine.score_pair(V[0], V[1], 0.6, 15.0, precision)
    assert r["status"] == 0 and r["B"] == 63
    for key, printed in (("mic", 0.999999), ("mas", 0.728144), ("mev", 0.999999),
                         ("mcn", 4.584963)):
        assert abs(r[key] - printed) <= 5e-7, (key, r[key])
    assert r["mcn_xy"] == 24


def test_config1_fp64_every_task():
    V, P = workloads.config1()
    run = run_batch(V, P, 0.6, 15.0, gmine.PLAIN_FP64)
    checked, differ = compare_tasks(V, P, run, range(P.shape[0]), 0.6, 15.0)
    assert checked == 16 * 2 * 14 and differ == 0
    compare_pairs(V, P, run, 0.6, 15.0, FP64_TOL)


def test_config1_fp32_rescored():
    V, P = workloads.config1()
    run = run_batch(V, P, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE)
    checked, differ = compare_tasks(V, P, run, range(P.shape[0]), 0.6, 15.0,
                                    check_cuts=False, I_tol=1e-5)
    print("config1 fp32: tasks %d, chosen partitions differing %d" % (checked, differ))
    compare_pairs(V, P, run, 0.6, 15.0, FP32_TOL)


def test_config2_fp64_all_pairs():
    V, P = workloads.config2()
    run = run_batch(V, P, 0.6, 15.0, gmine.PLAIN_FP64)
    errs = compare_pairs(V, P, run, 0.6, 15.0, FP64_TOL)
    rng = np.random.default_rng(0)
    sample = rng.choice(P.shape[0], 40, replace=False)
    checked, differ = compare_tasks(V, P, run, sample, 0.6, 15.0)
    assert differ == 0
    print("config2 fp64 max errors", errs)


def test_config2_fp32_all_pairs():
    V, P = workloads.config2()
    run = run_batch(V, P, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE)
    errs = compare_pairs(V, P, run, 0.6, 15.0, FP32_TOL)
    rng = np.random.default_rng(1)
    sample = rng.choice(P.shape[0], 40, replace=False)
    checked, differ = compare_tasks(V, P, run, sample, 0.6, 15.0, check_cuts=False, I_tol=1e-5)
    print("config2 fp32 max errors", errs, "partitions differing %d of %d" % (differ, checked))


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_ties_and_edge_cases(precision):
    tol = FP64_TOL if precision == gmine.PLAIN_FP64 else FP32_TOL
    T, P = workloads.tie_heavy(p=8, n=400, levels=6)
    rng = np.random.default_rng(9)
    extra = np.stack([
        np.ones(400),                                  # constant
        rng.normal(size=400),
        np.repeat(np.arange(4.0), 100),                # four big ties
        np.where(np.arange(400) < 3, 0.0, 1.0),        # nearly constant
    ])
    V = np.concatenate([T, extra])
    p = V.shape[0]
    P = np.concatenate([P, np.array([[8, 9], [9, 8], [10, 9], [11, 9], [10, 11], [9, 9]],
                                    dtype=np.int32)])
    run = run_batch(V, P, 0.6, 15.0, precision)
    compare_pairs(V, P, run, 0.6, 15.0, tol)
    checked, differ = compare_tasks(V, P, run, range(P.shape[0]), 0.6, 15.0,
                                    check_cuts=precision == gmine.PLAIN_FP64,
                                    I_tol=1e-9 if precision == gmine.PLAIN_FP64 else 1e-5)
    s = run["scores"]
    assert s["status"][P.shape[0] - 6] == gmine.E_CONSTANT
    assert p == 12


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_missing_samples_dropped_per_pair(precision):
    tol = FP64_TOL if precision == gmine.PLAIN_FP64 else FP32_TOL
    V, P, alphas, ns = workloads.config4(n_pairs=24, n_lo=20, n_hi=1500)
    run = run_batch(V, P, 0.6, 15.0, precision)
    compare_pairs(V, P, run, 0.6, 15.0, tol)
    checked, differ = compare_tasks(V, P, run, range(P.shape[0]), 0.6, 15.0,
                                    check_cuts=precision == gmine.PLAIN_FP64,
                                    I_tol=1e-9 if precision == gmine.PLAIN_FP64 else 1e-5)
    assert checked > 0


def test_errors_and_empty():
    import torch
    V, P = workloads.config1()
    Vd = torch.from_numpy(V).cuda()
    bad = torch.tensor([[0, 1], [0, 99], [-1, 2]], dtype=torch.int32, device="cuda")
    scores, M = gmine.compute_batch(Vd, bad, 0.6, 15.0)
    torch.cuda.synchronize()
    s = gmine.scores_to_numpy(scores)
    assert s["status"].tolist() == [gmine.OK, gmine.E_ARG, gmine.E_ARG]
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    scores, M = gmine.compute_batch(Vd, empty, 0.6, 15.0)
    assert scores.shape[0] == 0
    with pytest.raises(gmine.GmineError) as ei:
        gmine.compute_batch(Vd, bad, 1.5, 15.0)
    assert ei.value.status == gmine.E_PARAM
    few = gmine.score_pair(np.arange(3.0), np.arange(3.0))
    assert few["status"] == gmine.E_TOO_FEW


def test_host_buffers_match_device_path():
    import torch
    V, P = workloads.config1()
    run = run_batch(V, P, 0.6, 15.0, gmine.PLAIN_FP64, trace=False)
    s_host, M_host = gmine.compute_batch_host(V, P, 0.6, 15.0, gmine.PLAIN_FP64)
    for key in ("mic", "mas", "mev", "mcn", "status", "mcn_xy", "n_used", "B", "m_cells"):
        assert np.array_equal(s_host[key], run["scores"][key]), key
    assert np.array_equal(M_host, run["M"])


def test_largest_n_single_pair():
    """The largest n sorted in shared memory (16384 samples per variable, B = 337)."""
    rng = np.random.default_rng(12)
    n = 16384
    x = rng.uniform(size=n)
    y = np.sin(6 * x) + 0.4 * rng.normal(size=n)
    ref = oracle.score_pair(x, y, 0.6, 15.0)
    for precision, tol in ((gmine.PLAIN_FP64, FP64_TOL), (gmine.FP32_DP_FP64_RESCORE, FP32_TOL)):
        r = gmine.score_pair(x, y, 0.6, 15.0, precision)
        assert r["status"] == ref["status"] and r["B"] == ref["B"] == 337
        for key in ("mic", "mas", "mev"):
            assert abs(r[key] - ref[key]) <= tol, (precision, key)
        assert np.max(np.abs(r["M"] - ref["M"])) <= tol
