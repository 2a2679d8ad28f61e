"""The timing and counting fields of gmine_trace (the ones bench.py builds its
roofline line and step breakdown from): the DP launch times, the per-stage
times and the counters are filled, consistent with each other and with a
CUDA-event time around the whole call, and asking for them does not change
the scores."""
import numpy as np
import pytest

from paper_1208_4271_gb300 import gmine, workloads


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_trace_timing_fields_are_consistent(precision):
    import torch
    V, P = workloads.config3(p=30, n=1340)
    dev = torch.device("cuda:0")
    Vd = torch.from_numpy(V).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    ws = gmine.Workspace(V.shape[0], V.shape[1], P.shape[0], 0.6, 15.0, precision, device=dev)
    plain, _ = gmine.compute_batch(Vd, Pd, 0.6, 15.0, precision, want_M=False, workspace=ws)
    torch.cuda.synchronize()
    m = gmine.Measure(device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    timed, _ = gmine.compute_batch(Vd, Pd, 0.6, 15.0, precision, want_M=False, workspace=ws,
                                   trace=m.trace)
    e1.record()
    torch.cuda.synchronize()
    wall = e0.elapsed_time(e1)
    # the same scores with and without the trace
    a, b = gmine.scores_to_numpy(plain), gmine.scores_to_numpy(timed)
    for k in ("status", "mic", "mas", "mev", "mcn"):
        assert np.array_equal(a[k], b[k]), k
    # one time per DP launch of the plan, summing to the DP total
    groups = gmine.dp_groups(V.shape[1], 0.6, 15.0, precision)
    assert m.dp_launches == len(groups)
    lm = m.launch_ms
    assert lm.shape == (len(groups),) and np.all(lm > 0)
    assert abs(float(lm.sum()) - m.dp_ms) <= 1e-3 * m.dp_ms + 1e-3
    # stages: all present, non-negative, the DP stage covers the DP launches,
    # and together they fit inside the call's own time
    st = m.stage_ms
    assert set(st) == set(gmine.STAGE_NAMES)
    assert all(v >= 0.0 for v in st.values())
    assert st["dp"] >= 0.99 * m.dp_ms and st["partition"] > 0.0
    assert sum(st.values()) <= wall * 1.01 + 0.05
    # counters: the closed-form DP candidate count is positive, tasks = every
    # (pair, orientation, row count) the DP ran
    cand, tasks = (int(x) for x in m.counters.cpu())
    assert cand > 0
    B = gmine.B_of(V.shape[1], 0.6)
    assert tasks == 2 * P.shape[0] * (B // 2 - 1)
    assert m.kernel_launches >= len(groups) + 4
