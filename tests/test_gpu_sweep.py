"""The parameter sweeps on the GPU: the c sweep's MIC against the oracle at
c far from the default (small c: many superclump merges; large c: none) in
both precisions, and a small scaling run."""
import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import gmine, sweep, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    gmine.lib()


def test_c_sweep_matches_oracle():
    # c = 120: the row counts with four levels (split by x) all take the
    # blocked kernel's 4-level instance, with different shared-memory plans
    cs = [1.0, 2.0, 50.0, 120.0]
    recs = sweep.c_sweep(cs, n=675, n_pairs=3, alpha=0.551)
    S, Q = workloads.sparse_count_pairs(675, 3)
    ref = {c: oracle.score_batch(S, Q, 0.551, c)["stats"][:, 0] for c in cs}
    seen = 0
    for r in recs:
        if r["sweep"] != "c":
            continue
        tol = 1e-9 if r["precision"] == "fp64" else 1e-4
        assert np.max(np.abs(np.array(r["mic"]) - ref[r["c"]])) <= tol, r
        seen += 1
    assert seen == 2 * len(cs)
    conv = [r for r in recs if r["sweep"] == "c_convergence"]
    assert len(conv) == 2 * len(cs)
    assert all(r["max_abs_diff_to_c_max"] == 0.0 for r in conv if r["c"] == 120.0)


def test_time_sweep_small():
    recs = sweep.time_sweep([300], [0.6, 0.7], reps=8, repeats=1)
    times = [r for r in recs if r["sweep"] == "time"]
    assert len(times) == 4 and all(r["ms_per_pair"] > 0 for r in times)
    ratios = [r for r in recs if r["sweep"] == "time_ratio"]
    assert len(ratios) == 2 and all(r["ratio_06_07"] > 0 for r in ratios)
