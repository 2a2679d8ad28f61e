"""The parameter-sweep tool (SI Sec. 2C scaling; the c-convergence figure)
without a GPU: its plans, its seeded inputs, and the premise of the c sweep
checked on the oracle (once k-hat exceeds every clump count, the superclump
step never runs and MIC no longer depends on c)."""
import json
import subprocess
import sys
import os

import numpy as np

import oracle
from paper_1208_4271_gb300 import sweep, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_dry_run_plans():
    r = subprocess.run([sys.executable, "-m", "paper_1208_4271_gb300.sweep", "time", "--sizes", "250,500",
                        "--alphas", "0.5,0.6,0.7", "--precision", "fp32", "--dry-run"],
                       cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    recs = [json.loads(l) for l in r.stdout.splitlines()]
    assert len(recs) == 6 and {x["n"] for x in recs} == {250, 500}
    assert sweep.c_plan([1.0, 15.0], ["fp64", "fp32"]) == [
        {"sweep": "c", "c": 1.0, "precision": "fp64"}, {"sweep": "c", "c": 1.0, "precision": "fp32"},
        {"sweep": "c", "c": 15.0, "precision": "fp64"}, {"sweep": "c", "c": 15.0, "precision": "fp32"}]


def test_inputs_are_seeded_and_shaped():
    V1, P1 = workloads.uniform_pairs(300, 5)
    V2, _ = workloads.uniform_pairs(300, 5)
    assert V1.shape == (10, 300) and P1.tolist() == [[0, 1], [2, 3], [4, 5], [6, 7], [8, 9]]
    assert np.array_equal(V1, V2) and V1.min() >= 0.0 and V1.max() < 1.0
    assert not np.array_equal(V1[:, :10], workloads.uniform_pairs(301, 5)[0][:, :10])
    S, Q = workloads.sparse_count_pairs(675, 4)
    assert S.shape == (8, 675) and Q.shape == (4, 2)
    assert (S == 0).mean() > 0.3                       # many absent taxa: heavy ties
    assert np.all(S == np.round(S)) and S.min() >= 0.0


def test_mic_stops_depending_on_c_once_superclumps_vanish():
    S, Q = workloads.sparse_count_pairs(675, 3)
    alpha = 0.551
    x, y = S[Q[1, 0]], S[Q[1, 1]]
    big = [oracle.score_pair(x, y, alpha, c)["mic"] for c in (700.0, 1400.0)]
    # k-hat = c * floor(B / y) >= 700 > n = 675 >= clumps for every task
    assert big[0] == big[1]
    small = oracle.score_pair(x, y, alpha, 1.0)["mic"]
    assert 0.0 <= small <= 1.0
