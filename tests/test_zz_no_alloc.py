"""gmine_compute_batch_static, the batch call that allocates nothing, against
the ordinary workspace call (gmine_compute_batch).

The static call is for callers that cannot allocate device memory (a host
application that keeps all GPU memory in its own pool, or a latency-critical
path that cannot take cudaMalloc's device-wide synchronisation): its scratch
is a fixed array inside the library.  Two calls in a row must both give the
ordinary call's results, since the array keeps the previous call's contents.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1208_4271_gb300 import gmine, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_static_scratch_matches_workspace_call(precision):
    torch = _cuda()
    V, P = workloads.config1()
    Vd = torch.from_numpy(V).cuda()
    Pd = torch.from_numpy(P).cuda()
    ref_scores, ref_M = gmine.compute_batch(Vd, Pd, 0.6, 15.0, precision, want_M=True)
    torch.cuda.synchronize()
    ref = gmine.scores_to_numpy(ref_scores)
    ref_M = ref_M.cpu().numpy()
    for call in range(2):
        rc, scores, M = gmine.compute_batch_static(Vd, Pd, 0.6, 15.0, precision, want_M=True)
        torch.cuda.synchronize()
        assert rc == gmine.OK, gmine.strerror(rc)
        got = gmine.scores_to_numpy(scores)
        for key in ("status", "n_used", "B", "m_cells", "mcn_xy", "yhat_x", "yhat_y"):
            assert np.array_equal(got[key], ref[key]), (call, key)
        for key in ("mic", "mas", "mev", "mcn"):
            assert np.max(np.abs(got[key] - ref[key])) <= TOL, (call, key)
        assert np.max(np.abs(M.cpu().numpy() - ref_M)) <= TOL, call


def test_static_scratch_refuses_batches_above_its_size():
    torch = _cuda()
    V, P = workloads.config2()          # 4950 pairs at n = 1000: far above 64 MiB
    Vd = torch.from_numpy(V).cuda()
    Pd = torch.from_numpy(P).cuda()
    rc, scores, M = gmine.compute_batch_static(Vd, Pd, 0.6, 15.0, gmine.PLAIN_FP64, want_M=False)
    torch.cuda.synchronize()
    assert rc == gmine.E_WORKSPACE
    assert int(scores.sum(dtype=torch.int64).item()) == 0     # nothing was written
