"""The DP plan autotuner (paper_1208_4271_gb300/tune.py) on CPU with a fake
backend: it keeps the fastest candidate the library accepts for each launch
group, skips candidates that do not apply or change the scores, leaves the
chosen set active, and its cache file merges and applies per device.  The
GPU test runs it on the device: every chosen plan fits shared memory and a
tuned batch still matches the oracle."""
import json

import numpy as np
import pytest

from paper_1208_4271_gb300 import gmine, tune


class FakeBackend:
    """Two launch groups; `feasible` lists the (kind, threads) each group
    accepts, `ms` their times; one candidate gives different scores."""

    def __init__(self):
        self.shape = (1340, 0.6, 15.0, gmine.FP32_DP_FP64_RESCORE)
        self.device_name = "fake-gpu"
        self.default = [dict(ylo=2, yhi=2, kind=gmine.DP_BLOCKED, threads=256, smem=100, lev=36),
                        dict(ylo=10, yhi=12, kind=gmine.DP_BLOCKED, threads=128, smem=50, lev=8)]
        self.feasible = [{(gmine.DP_BLOCKED, 128): 1.5, (gmine.DP_BLOCKED, 256): 2.0,
                          (gmine.DP_MID, 256): 1.2},
                         {(gmine.DP_BLOCKED, 128): 1.0, (gmine.DP_BLOCKED, 256): 0.9,
                          (gmine.DP_WARP, 64): 0.7, (gmine.DP_SMALL, 32): 0.1}]
        self.wrong = (1, (gmine.DP_SMALL, 32))  # fastest, but gives other scores
        self.choices = []
        self.sets = []

    def set_choices(self, choices):
        self.choices = [dict(c) for c in choices]
        self.sets.append(self.choices)

    def groups(self):
        out = [dict(g) for g in self.default]
        for c in self.choices:
            for gi, g in enumerate(out):
                if (g["ylo"], g["yhi"]) == (c["ylo"], c["yhi"]) and \
                        (c["kind"], c["threads"]) in self.feasible[gi]:
                    g["kind"], g["threads"] = c["kind"], c["threads"]
        return out

    def run(self):
        eff = self.groups()
        ms = np.array([self.feasible[gi][(g["kind"], g["threads"])] for gi, g in enumerate(eff)])
        s = np.zeros(4, dtype=gmine.SCORE_DTYPE)
        s["mic"] = 0.5
        if (eff[self.wrong[0]]["kind"], eff[self.wrong[0]]["threads"]) == self.wrong[1]:
            s["mic"][2] += 1e-6
        return ms, s


def test_tuner_keeps_fastest_valid_candidate():
    be = FakeBackend()
    e = tune.tune(be)
    got = [(g["kind"], g["threads"]) for g in e["groups"]]
    # group 0: the level-major shape at 1.2 ms beats both blocked sizes;
    # group 1: the warp shape (0.7 ms); the small shape is faster but wrong
    assert got == [(gmine.DP_MID, 256), (gmine.DP_WARP, 64)]
    assert e["groups"][0]["default_ms"] == 2.0 and e["groups"][1]["ms"] == 0.7
    assert any(t[2] is None for t in e["groups"][1]["tried"])       # the rejected one
    assert be.choices == [{f: g[f] for f in ("ylo", "yhi", "kind", "threads")} for g in e["groups"]]
    assert e["device"] == "fake-gpu" and e["n"] == 1340 and e["precision"] == 1


def test_candidates_cover_the_kernel_shapes():
    two = tune.candidates(dict(ylo=30, yhi=37), 75, True)
    assert (gmine.DP_TWO, 256) in two and (gmine.DP_SMALL, 32) in two
    big = tune.candidates(dict(ylo=2, yhi=2), 75, True)
    kinds = {k for k, _ in big}
    assert gmine.DP_TWO not in kinds and gmine.DP_SMALL not in kinds and gmine.DP_WARP in kinds
    assert gmine.DP_WARP not in {k for k, _ in tune.candidates(dict(ylo=2, yhi=2), 75, False)}


def test_cache_merge_and_apply_per_device(tmp_path):
    path = str(tmp_path / "tuned.json")
    e1 = tune.tune(FakeBackend())
    tune.save(e1, path)
    e2 = dict(e1, device="other-gpu")
    tune.save(e2, path)
    tune.save(e1, path)                                    # replaces, does not duplicate
    entries = tune.load(path)
    assert len(entries) == 2
    assert json.load(open(path)) == entries
    calls = []
    k = tune.apply(entries, device_name="fake-gpu", setter=lambda *a: calls.append(a))
    assert k == 1 and len(calls) == 1
    n, alpha, c, prec, ch = calls[0]
    assert (n, alpha, c, prec) == (1340, 0.6, 15.0, 1)
    assert [(g["kind"], g["threads"]) for g in ch] == [(gmine.DP_MID, 256), (gmine.DP_WARP, 64)]
    assert tune.apply(entries, device_name="absent", setter=lambda *a: calls.append(a)) == 0
    assert tune.load(str(tmp_path / "none.json")) == []
    # a group whose best was the planner's own choice stays with the rules
    e3 = dict(e1, device="third-gpu", groups=[dict(e1["groups"][0]), dict(e1["groups"][1])])
    e3["groups"][0].update(kind=e3["groups"][0]["default_kind"], threads=e3["groups"][0]["default_threads"])
    calls.clear()
    assert tune.apply([e3], device_name="third-gpu", setter=lambda *a: calls.append(a)) == 1
    assert [(g["kind"], g["threads"]) for g in calls[0][4]] == [(gmine.DP_WARP, 64)]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE])
def test_tuner_on_device_fits_and_keeps_parity(precision):
    import torch
    import oracle
    from paper_1208_4271_gb300 import workloads
    from gpu_util import compare_pairs, run_batch
    n, alpha, c = 1000, 0.6, 15.0
    be = tune.GpuBackend(n, alpha, c, precision, n_vars=24, reps=1)
    try:
        e = tune.tune(be)
        optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)
        groups = gmine.dp_groups(n, alpha, c, precision)
        assert [(g["kind"], g["threads"]) for g in groups] == \
            [(g["kind"], g["threads"]) for g in e["groups"]]
        for g in groups:
            assert g["smem"] + 1024 <= optin, g
        V, P = workloads.config2()
        idx = np.random.default_rng(9).choice(P.shape[0], 120, replace=False)
        run = run_batch(V, P[idx], alpha, c, precision, trace=False)
        compare_pairs(V, P[idx], run, alpha, c, 1e-9 if precision == gmine.PLAIN_FP64 else 1e-4)
    finally:
        gmine.set_dp_choices(n, alpha, c, precision, [])
