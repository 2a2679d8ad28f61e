"""Parity of the linear statistics reported beside MINE (Pearson rho and the
non-linearity index MIC - rho^2, Fig. 1; reading R11) and of the
master-variable (one-versus-all) pair lists the paper's large analyses use
(Table 1; SI Sec. 3A), through the C ABI against the FP64 oracle.

Tolerance of rho: both sides are two-pass FP64 sums over the same samples
and differ only in the order of the additions; for n <= 2,000 samples of
well-conditioned data that moves rho by a few units of 1e-16 per sample at
most, so 1e-11 absolute leaves a wide margin and still catches any wrong
term (a wrong mean, a dropped sample, a missing square root)."""
import math

import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import gmine, workloads

from gpu_util import run_batch

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    gmine.lib()


def _gpu_linear(V, P, scores=None):
    import torch
    Vd = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).cuda()
    Pd = torch.from_numpy(np.ascontiguousarray(P, dtype=np.int32)).cuda()
    sd = None
    if scores is not None:
        sd = torch.from_numpy(np.ascontiguousarray(scores).view(np.uint8).reshape(len(scores), -1)).cuda()
    rho, nl = gmine.pearson_batch(Vd, Pd, sd)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), (nl.cpu().numpy() if nl is not None else None)


def _check_rho(V, P, rho):
    for i, (a, b) in enumerate(P):
        r, _ = oracle.pearson(V[a], V[b])
        if math.isnan(r):
            assert math.isnan(rho[i]), i
        else:
            assert abs(rho[i] - r) <= RHO_TOL, (i, rho[i], r)


def test_pearson_parity_config2_all_pairs():
    V, P = workloads.config2()
    rho, _ = _gpu_linear(V, P)
    assert rho.shape == (P.shape[0],)
    _check_rho(V, P, rho)


def test_pearson_missing_ties_and_degenerate_pairs():
    rng = np.random.default_rng(31)
    n = 777  # a ragged tail over the 32 lanes
    V = rng.lognormal(5.0, 1.2, size=(8, n))
    V[1] = np.round(V[0] / 40.0) * 40.0 + rng.normal(scale=5.0, size=n)  # ties
    V[2] = 3.0                                    # constant: rho undefined
    V[3, ::3] = np.nan                            # missing samples
    V[4, 5::7] = np.inf
    V[5] = np.nan
    V[5, :1] = 1.0                                # one finite sample
    V[6] = -2.0 * V[0] + 1.0                      # exact line: rho = -1
    V[7, ::2] = np.nan
    P = workloads.all_pairs(8)
    rho, _ = _gpu_linear(V, P)
    _check_rho(V, P, rho)
    i = [k for k, (a, b) in enumerate(P) if (a, b) == (0, 6)][0]
    assert abs(rho[i] + 1.0) <= 1e-14
    for k, (a, b) in enumerate(P):
        if 2 in (a, b) or 5 in (a, b):
            assert math.isnan(rho[k])


def test_pearson_out_of_range_pair_gives_nan():
    V, _ = workloads.config1()
    P = np.array([[0, 1], [0, V.shape[0]], [-1, 2]], dtype=np.int32)
    rho, _ = _gpu_linear(V, P)
    assert abs(rho[0] - oracle.pearson(V[0], V[1])[0]) <= RHO_TOL
    assert math.isnan(rho[1]) and math.isnan(rho[2])


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_nonlinearity_index_parity(precision):
    V, P = workloads.config1()
    run = run_batch(V, P, precision=precision, trace=False, want_M=False)
    sc = run["scores"]
    rho, nl = _gpu_linear(V, P, sc)
    ref = oracle.score_batch(V, P)
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    for i, (a, b) in enumerate(P):
        r, _ = oracle.pearson(V[a], V[b])
        expect = oracle.nonlinearity(ref["stats"][i, 0], r)
        assert abs(nl[i] - expect) <= tol + 2 * RHO_TOL, (i, nl[i], expect)
        # the device value is MIC - rho^2 of the device's own MIC and rho
        assert nl[i] == sc["mic"][i] - rho[i] * rho[i]


def test_nonlinearity_nan_for_invalid_pairs():
    rng = np.random.default_rng(32)
    V = rng.normal(size=(3, 50))
    V[2, 3:] = np.nan  # 3 finite samples: MINE status E_TOO_FEW, rho defined
    P = np.array([[0, 1], [0, 2]], dtype=np.int32)
    run = run_batch(V, P, trace=False, want_M=False)
    assert run["scores"]["status"][1] != gmine.OK
    rho, nl = _gpu_linear(V, P, run["scores"])
    assert not math.isnan(rho[1]) and math.isnan(nl[1])
    assert not math.isnan(nl[0])


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_master_variable_pairs(precision):
    """One variable against all others (the paper's 1-vs-all analyses): the
    master's ranks and row maps are shared by all its pairs; every score
    matches the oracle and, bit for bit, the same pair inside an all-pairs
    batch."""
    V, _ = workloads.config2()
    V = V[:40]
    master = 7
    P = np.array([[master, j] for j in range(V.shape[0]) if j != master], dtype=np.int32)
    run = run_batch(V, P, precision=precision, trace=False, want_M=True)
    ref = oracle.score_batch(V, P)
    tol = 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4
    for s, key in enumerate(("mic", "mas", "mev", "mcn")):
        assert np.max(np.abs(run["scores"][key] - ref["stats"][:, s])) <= tol
    Pall = workloads.all_pairs(V.shape[0])
    Pall = np.concatenate([Pall, Pall[:, ::-1]]).astype(np.int32)  # both orders
    allrun = run_batch(V, Pall, precision=precision, trace=False, want_M=False)
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(Pall)}
    for i, (a, b) in enumerate(P):
        j = index[(int(a), int(b))]
        for key in ("mic", "mas", "mev", "mcn", "status", "n_used"):
            assert run["scores"][key][i] == allrun["scores"][key][j], (key, a, b)
