"""Parity at the largest sizes of the workloads, both precisions, against the oracle.

* n = 100,000 samples at alpha = 0.6 (B = 999: up to 7,485 superclumps per
  task, 498 row counts per orientation, 5,056 cells): a heavy-tie pair from
  the negative-binomial count generator, a continuous pair with small noise
  and a noiseless monotone pair.  The plain FP64 path matches the oracle's
  statistics and every cell of M to 1e-9 with the same MCN cell, and the
  integer quantities of sampled tasks (yhat, clump count, superclump ends,
  chosen partitions) bit for bit; the FP32 path is within 1e-4.
* alpha = 0.75: a rounded pair at n = 20,000 (B = 1,681) and uneven pairs
  with missing samples (n up to 6,000), both precisions.

The oracle's results come from a background thread started at collection
(tests/large_cases.py), so that its minutes of CPU time overlap the GPU tests
that run first.
"""
import numpy as np
import pytest

from paper_1208_4271_gb300 import gmine

import large_cases
from gpu_util import compare_pairs, run_batch, task_index

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_n100000_against_oracle(precision):
    V, P, alpha = large_cases.case("n100k")
    plain = precision == gmine.PLAIN_FP64
    tol = 1e-9 if plain else 1e-4
    run = run_batch(V, P, alpha, large_cases.C, precision, trace=plain, want_M=True)
    s = run["scores"]
    assert np.all(s["B"] == 999) and np.all(s["m_cells"] == 5056)
    ref = large_cases.oracle_pairs("n100k")
    errs = compare_pairs(V, P, run, alpha, large_cases.C, tol, ref=ref)
    print("n = 100000 precision %d: %s" % (precision, errs))
    if not plain:
        return
    tr = run["trace"]
    for (i, o, y), want in large_cases.oracle_tasks("n100k").items():
        t = task_index(i, o, y, P.shape[0])
        k = want["k"]
        assert tr["yhat"][t] == want["yhat"], (i, o, y)
        assert tr["clumps"][t] == want["clumps"], (i, o, y)
        assert tr["k"][t] == k, (i, o, y, tr["k"][t], k)
        assert np.array_equal(tr["sc_ends"][t, :k + 1], want["sc_ends"]), (i, o, y)
        x = want["x"]
        assert np.max(np.abs(tr["I"][t, :x - 1] - want["I"])) <= 1e-9, (i, o, y)
        for l in range(2, x + 1):
            off = (l - 2) * (l - 1) // 2
            assert tr["cuts"][t, off:off + l - 1].tolist() == want["cuts"][l - 2], (i, o, y, l)


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_alpha_075_against_oracle(precision):
    V, P, alpha = large_cases.case("a075")
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    run = run_batch(V, P, alpha, large_cases.C, precision, trace=False, want_M=True)
    assert run["scores"]["B"][0] == 1681
    errs = compare_pairs(V, P, run, alpha, large_cases.C, tol, ref=large_cases.oracle_pairs("a075"))
    print("alpha = 0.75 precision %d: %s" % (precision, errs))
