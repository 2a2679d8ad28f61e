"""Every kernel shape of the OptimizeXAxis DP gives the same scores.

The planner sends each launch group (a range of row counts y) to one of
five kernels (blocked CTA per task, warp per task, level-major, small-x,
two-column) and picks a CTA size; the autotuner may pick another.  They
compute the same recursion (SOM Algorithm 2, Appendix item 10) in other
orders of the same exact maxima, so on the plain FP64 path every shape must
give bit-identical scores and M, and on the float path the same scores to
within the re-score's summation order (1e-9).  Each feasible (shape, CTA
size) of each group is forced in turn through gmine_set_dp_choices and
compared with the planner's own choice, on config-3-shaped data and on
heavy-tie data (ties change the clump and superclump structure)."""
import numpy as np
import pytest

from paper_1208_4271_gb300 import gmine, tune, workloads
from gpu_util import run_batch

N, ALPHA, C = 1340, 0.6, 15.0


def _data(kind):
    if kind == "config3":
        return workloads.config3(p=24, n=N)
    V, P = workloads.config5(p=24, n=N)
    return V, P


def _same(a, b, exact):
    sa, sb = a["scores"], b["scores"]
    assert np.array_equal(sa["status"], sb["status"])
    for k in ("mic", "mas", "mev"):
        if exact:
            assert np.array_equal(sa[k], sb[k]), k
        else:
            assert np.max(np.abs(sa[k] - sb[k]), initial=0.0) <= 1e-9, k
    if exact:
        assert np.array_equal(a["M"], b["M"])
    else:
        assert np.max(np.abs(a["M"] - b["M"]), initial=0.0) <= 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("data", ["config3", "ties"])
@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_every_kernel_shape_gives_the_same_scores(precision, data):
    V, P = _data(data)
    fp32 = precision == gmine.FP32_DP_FP64_RESCORE
    B = gmine.B_of(N, ALPHA)
    gmine.set_dp_choices(N, ALPHA, C, precision, [])
    try:
        ref = run_batch(V, P, ALPHA, C, precision, trace=False)
        groups = gmine.dp_groups(N, ALPHA, C, precision)
        tried = 0
        for gi, g in enumerate(groups):
            for kind, threads in tune.candidates(g, B, fp32):
                if (kind, threads) == (g["kind"], g["threads"]):
                    continue
                choice = {"ylo": g["ylo"], "yhi": g["yhi"], "kind": kind, "threads": threads}
                gmine.set_dp_choices(N, ALPHA, C, precision, [choice])
                eff = gmine.dp_groups(N, ALPHA, C, precision)
                if len(eff) != len(groups) or (eff[gi]["kind"], eff[gi]["threads"]) != (kind, threads):
                    continue  # not feasible for this group
                got = run_batch(V, P, ALPHA, C, precision, trace=False)
                _same(ref, got, exact=not fp32)
                tried += 1
        # every group has at least one other feasible CTA size or shape
        assert tried >= len(groups)
    finally:
        gmine.set_dp_choices(N, ALPHA, C, precision, [])
