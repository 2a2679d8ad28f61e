"""Parity at the benchmark's full size and on the other workload shapes.

* all 1,999,000 pairs of 2000 variables x n = 1340 (the metric's workload), in
  the launch configuration bench.py times (one gmine_compute_batch, FP32 DP
  with FP64 re-score): sampled pairs against the oracle, MIC/MAS/MEV <= 1e-4;
  every pair: valid status, 0 <= M-statistics <= 1, MCN = log2(mcn_xy);
* the plain FP64 path on the bench's FP64 subset (all pairs of 200
  variables): sampled pairs to 1e-9 with exact MCN cells and chosen
  partitions on sampled tasks;
* heavy ties (negative-binomial counts, log2(c+1)) and uneven pairs with
  missing samples at alpha in {0.55, 0.6, 0.75}: every pair, FP64 and FP32.
"""
import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import gmine, workloads

from gpu_util import compare_pairs, compare_tasks, run_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def config3_full():
    return workloads.config3(p=2000, n=1340)


def test_metric_workload_full_size_fp32_sampled(config3_full):
    import torch
    V, P = config3_full
    assert P.shape[0] == 1999000
    Vd = torch.from_numpy(V).cuda()
    Pd = torch.from_numpy(P).cuda()
    scores, _ = gmine.compute_batch(Vd, Pd, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE, want_M=False)
    torch.cuda.synchronize()
    s = gmine.scores_to_numpy(scores)
    assert np.all(s["status"] == gmine.OK)
    assert np.all(s["n_used"] == 1340) and np.all(s["B"] == 75) and np.all(s["m_cells"] == 189)
    for key in ("mic", "mas", "mev"):
        assert np.all(s[key] >= 0.0) and np.all(s[key] <= 1.0 + 1e-9)
    assert np.all(s["mev"] <= s["mic"])
    assert np.allclose(s["mcn"], np.log2(s["mcn_xy"]), rtol=0, atol=1e-12)
    rng = np.random.default_rng(2012)
    idx = np.sort(rng.choice(P.shape[0], 96, replace=False))
    ref = oracle.score_batch(V, P[idx], 0.6, 15.0, nthreads=0)
    got = np.stack([s["mic"][idx], s["mas"][idx], s["mev"][idx]], axis=1)
    err = np.abs(got - ref["stats"][:, :3]).max(axis=0)
    print("full-size FP32 sample: max |err| MIC %.2e MAS %.2e MEV %.2e" % tuple(err))
    assert np.all(err <= 1e-4)


def test_bench_fp64_subset_sampled(config3_full):
    V, P = config3_full
    sub = 200
    Ps = workloads.all_pairs(sub)
    run = run_batch(V[:sub], Ps, 0.6, 15.0, gmine.PLAIN_FP64, trace=True, want_M=True)
    rng = np.random.default_rng(2013)
    idx = np.sort(rng.choice(Ps.shape[0], 48, replace=False))
    compare_pairs(V[:sub], Ps, run, 0.6, 15.0, 1e-9, idx=idx)
    checked, differ = compare_tasks(V[:sub], Ps, run, idx[:6], 0.6, 15.0)
    assert checked > 0 and differ == 0


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_heavy_ties_negative_binomial(precision):
    V, P = workloads.config5(p=40, n=1340)
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    run = run_batch(V, P, 0.6, 15.0, precision)
    compare_pairs(V, P, run, 0.6, 15.0, tol)
    rng = np.random.default_rng(5)
    sample = rng.choice(P.shape[0], 8, replace=False)
    checked, differ = compare_tasks(V, P, run, sample, 0.6, 15.0,
                                    check_cuts=precision == gmine.PLAIN_FP64,
                                    I_tol=1e-9 if precision == gmine.PLAIN_FP64 else 1e-5)
    assert checked > 0


@pytest.mark.parametrize("alpha", [0.55, 0.6, 0.75])
@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_uneven_pairs_with_missing_samples(alpha, precision):
    n_hi = 6000 if alpha <= 0.6 else 1500  # keeps the oracle at a few seconds
    V, P, _, ns = workloads.config4(n_pairs=40, n_lo=50, n_hi=n_hi, seed_salt=int(alpha * 100))
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    run = run_batch(V, P, alpha, 15.0, precision, trace=False)
    compare_pairs(V, P, run, alpha, 15.0, tol)


@pytest.fixture(scope="module")
def large_n_batch():
    # n = 20000 (the largest n of the uneven workload): a clean pair, a pair
    # whose second variable misses 15 % of the samples (compacted to about
    # 17,000), and a tie-heavy pair (rounded values); n > 16,384 takes the
    # sort and partition paths through global scratch
    rng = np.random.default_rng(20000)
    n = 20000
    x = rng.random(n)
    V = np.empty((6, n))
    V[0] = x
    V[1] = np.sin(6.0 * x) + 0.3 * rng.standard_normal(n)
    V[2] = rng.random(n)
    V[3] = V[2] ** 2 + 0.05 * rng.standard_normal(n)
    V[3][rng.random(n) < 0.15] = np.nan
    V[4] = np.round(rng.random(n) * 40.0)
    V[5] = np.round(V[4] + 3.0 * rng.standard_normal(n))
    P = np.array([[0, 1], [2, 3], [4, 5]], dtype=np.int32)
    ref = oracle.score_batch(V, P, 0.6, 15.0, nthreads=0, want_M=True)
    return V, P, ref


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_large_n_beyond_shared_memory_sort(large_n_batch, precision):
    V, P, ref = large_n_batch
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    run = run_batch(V, P, 0.6, 15.0, precision, trace=False)
    errs = compare_pairs(V, P, run, 0.6, 15.0, tol, ref=ref)
    print("n = 20000 precision %d: %s" % (precision, errs))


def test_n_100000_properties():
    """n = 100,000 (B = 999, up to 7,485 superclumps): the FP32 path, checked
    by properties that hold at any size (the oracle is too slow here): MIC = 1
    for a noiseless monotone pair, 0 <= M-statistics <= 1, MEV <= MIC,
    MCN = log2(mcn_xy), 5,056 cells, and bitwise-identical scores after a
    permutation of the samples (the oracle comparison at this size is in
    test_gpu_large.py)."""
    rng = np.random.default_rng(100000)
    n = 100000
    x = rng.random(n)
    V = np.stack([x, np.exp(3.0 * x), rng.random(n), np.zeros(n)])
    V[3] = np.sin(6.0 * V[2]) + 0.3 * rng.standard_normal(n)
    P = np.array([[0, 1], [2, 3]], dtype=np.int32)
    run = run_batch(V, P, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE, trace=False, want_M=True)
    s = run["scores"]
    assert np.all(s["status"] == gmine.OK)
    assert np.all(s["n_used"] == n) and np.all(s["B"] == 999) and np.all(s["m_cells"] == 5056)
    assert abs(s["mic"][0] - 1.0) <= 1e-9
    for key in ("mic", "mas", "mev"):
        assert np.all(s[key] >= 0.0) and np.all(s[key] <= 1.0 + 1e-9)
    assert np.all(s["mev"] <= s["mic"] + 1e-12)
    assert np.allclose(s["mcn"], np.log2(s["mcn_xy"]), rtol=0, atol=1e-12)
    perm = rng.permutation(n)
    run2 = run_batch(V[:, perm], P, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE, trace=False, want_M=True)
    for key in ("mic", "mas", "mev", "mcn"):
        assert np.array_equal(s[key], run2["scores"][key]), key
    assert np.array_equal(run["M"], run2["M"])
    print("n = 100000: MIC %.6f %.6f, MAS %.6f, MCN %.3f" % (s["mic"][0], s["mic"][1], s["mas"][1], s["mcn"][1]))
