"""Benchmark: MINE pairs/s at n = 1340, alpha = 0.6, c = 15 (all pairs of
2000 synthetic microarray-shaped variables, 1,999,000 pairs per step).

Our arm (default): the batched GB300 path through the libgmine C ABI, FP32
DP with FP64 re-scoring of each chosen partition (`value`), with the plain
FP64 DP measured beside it on a subset of the same pairs.  One step = one
whole gmine_compute_batch over every pair of the batch (ranks, equipartition,
clumps/superclumps, DP, M and the four statistics), inputs resident in HBM.

Reference arm (--impl reference): the FP64 CPU oracle on this host's cores,
each step a bounded sample of the same pairs.

One JSON line is printed by rank 0.  Under torchrun every rank computes its
own independently seeded copy of the workload (pairs are independent: weak
scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MINE pairs/sec at n=1340 α=0.6 c=15: batched FP32-DP vs plain FP64, same GPU"
ALPHA = 0.6
C = 15.0
N_SAMPLES = 1340
N_VARS = 2000
L2_FLUSH_BYTES = 256 << 20
# FP64 operations (thread instructions) an SM executes per clock on GB300:
# ncu reports sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained =
# 2 per SM and cycle (152 SMs x 2 x 2.07 GHz x 2 flops = the nominal 1.25
# TFLOP/s of FP64 FMA)
FP64_PER_SM_CLK = 2
# DRAM bytes (read + write) per DP task of the float DP launches, from the
# ncu launch list of the 60-variable case (profiles/launches_config3_60vars.md:
# 1,160 MB for 254,880 tasks); the launches read their task records and
# little else, so the traffic scales with the tasks
DP_DRAM_BYTES_PER_TASK = 4.55e3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmine", choices=["gmine", "reference"])
    ap.add_argument("--vars", type=int, default=N_VARS,
                    help="variables of the all-pairs workload (2000 = the metric's workload)")
    ap.add_argument("--fp64-vars", type=int, default=632,
                    help="variables whose all pairs time the plain FP64 path (632: 10 %% of "
                         "the metric workload's pairs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the uneven batch (20,000 pairs, n in [50, 20000], per-pair alpha)")
    ap.add_argument("--no-ties", action="store_true",
                    help="skip the heavy-tie batch (124,750 pairs at n=1340, 200 pairs at n=100000)")
    ap.add_argument("--uneven-pairs", type=int, default=20000)
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of the ranks' values (a step is as slow as the slowest
    rank); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def workload(rank, n_vars):
    from paper_1208_4271_gb300 import workloads
    V, P = workloads.config3(p=n_vars, n=N_SAMPLES, seed_salt=rank)
    return V, P


def oracle_sample(V, P, cpu_seconds, rng_seed=0, keep=None):
    """Time the FP64 CPU oracle on a bounded random sample of the pairs.

    With keep (a dict), the sampled pair indices and the oracle's statistics
    are stored in it for the parity report."""
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    probe = P[rng.choice(P.shape[0], min(P.shape[0], 2 * threads), replace=False)]
    t0 = time.perf_counter()
    oracle.score_batch(V, probe, ALPHA, C, nthreads=threads)
    rate = probe.shape[0] / max(time.perf_counter() - t0, 1e-6)
    m = int(min(P.shape[0], max(threads, rate * cpu_seconds)))
    idx = np.sort(rng.choice(P.shape[0], m, replace=False))
    sample = P[idx]
    t0 = time.perf_counter()
    ref = oracle.score_batch(V, sample, ALPHA, C, nthreads=threads)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep["idx"] = idx
        keep["stats"] = ref["stats"]
    return {"value": m / dt, "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "sample": "%d random pairs of the %d-variable all-pairs workload (n=%d), "
                      "FP64 oracle, OpenMP over pairs, %.1f s" % (m, V.shape[0], V.shape[1], dt)}


def error_summary(got, ref):
    """Max and 99th-percentile absolute error per statistic (MIC, MAS, MEV, MCN)."""
    out = {}
    for j, name in enumerate(("mic", "mas", "mev", "mcn")):
        e = np.abs(np.asarray(got[name], dtype=np.float64) - ref[:, j])
        out[name] = {"max": float(e.max()) if e.size else None,
                     "p99": float(np.percentile(e, 99)) if e.size else None}
    return out


def partition_flips(Vd, dev, nv):
    """Fraction of tasks whose chosen partition differs between the FP32 path
    and the plain FP64 path (whose partitions equal the oracle's), on all pairs
    of the first nv variables."""
    import torch
    from paper_1208_4271_gb300 import gmine
    Ps = torch.from_numpy(gmine_all_pairs(nv)).to(dev)
    cuts = {}
    for prec in (gmine.PLAIN_FP64, gmine.FP32_DP_FP64_RESCORE):
        tr, tt = gmine.alloc_trace(Ps.shape[0], Vd.shape[1], ALPHA, C, device=dev)
        gmine.compute_batch(Vd[:nv], Ps, ALPHA, C, prec, want_M=False, trace=tr)
        torch.cuda.synchronize(dev)
        cuts[prec] = (tt["k"].cpu().numpy(), tt["cuts"].cpu().numpy())
        del tt
    k64, c64 = cuts[gmine.PLAIN_FP64]
    k32, c32 = cuts[gmine.FP32_DP_FP64_RESCORE]
    live = (k64 >= 2) & (k32 == k64)
    differ = np.any(c64[live] != c32[live], axis=1)
    return {"tasks": int(live.sum()), "differing": int(differ.sum()),
            "fraction": float(differ.mean()) if live.any() else 0.0,
            "sample": "all %d pairs of the first %d variables" % (Ps.shape[0], nv)}


def oracle_errors(V, P, alphas, got, idx, threads):
    """Oracle statistics of the pairs idx and the largest absolute errors of
    the GPU's MIC, MAS, MEV (and MCN) on them."""
    import oracle
    ref = oracle.score_batch(V, P[idx], alphas if np.ndim(alphas) == 0 else alphas[idx], C,
                             nthreads=threads)
    ok = ref["status"] == 0
    out = {}
    for j, name in enumerate(("mic", "mas", "mev", "mcn")):
        e = np.abs(np.asarray(got[name][idx], dtype=np.float64) - ref["stats"][:, j])[ok]
        out[name] = float(e.max()) if e.size else None
    out["status_equal"] = bool(np.array_equal(np.asarray(got["status"][idx]), ref["status"]))
    return out


def bench_uneven(dev, args, threads, do_parity):
    """The uneven batch: 20,000 pairs with n log-uniform in [50, 20000], 0-20 %
    missing samples, alpha per pair in {0.55, 0.6, 0.75}, in one
    gmine_compute_batch_uneven call (FP32 DP, FP64 re-score), timed with CUDA
    events around the call (its planning read-back included).  Parity: the
    oracle on a random sample of the pairs whose DP work stays below a bound
    (the heaviest pairs take the oracle minutes each)."""
    import torch
    from paper_1208_4271_gb300 import gmine, workloads
    V, P, alphas, ns = workloads.config4(n_pairs=args.uneven_pairs)
    Vd = torch.from_numpy(V).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    prec = gmine.FP32_DP_FP64_RESCORE
    vals, _ = gmine.alpha_table(alphas)
    ws = gmine.UnevenWorkspace(V.shape[0], V.shape[1], P.shape[0], vals, C, prec, device=dev)
    meas = gmine.Measure(device=dev)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    scores, _ = gmine.compute_batch_uneven(Vd, Pd, alphas, C, prec, want_M=False, workspace=ws,
                                           measure=meas)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    s = gmine.scores_to_numpy(scores)
    out = {"value": P.shape[0] / (ms / 1e3), "unit": "pairs/s", "ms": ms,
           "workload": "%d pairs, n log-uniform in [50, 20000] (max %d), 0-20%% missing, "
                       "alpha per pair in {0.55, 0.6, 0.75}, c=15, one call" % (P.shape[0], int(ns.max())),
           "dp_candidates": int(meas.counters[0].item()), "dp_ms": meas.dp_ms,
           "dp_launches": meas.dp_launches, "gpu_launches": meas.kernel_launches}
    if meas.dp_ms > 0:
        out["dp_tcand_per_s"] = out["dp_candidates"] / (meas.dp_ms / 1e3) / 1e12
    del ws, Vd
    torch.cuda.empty_cache()
    if do_parity:
        rng = np.random.default_rng(44)
        light = np.flatnonzero(ns * np.where(alphas > 0.7, 4.0, 1.0) <= 3000)
        idx = np.sort(rng.choice(light, min(200, light.size), replace=False))
        t0 = time.perf_counter()
        out["fp32_vs_oracle"] = oracle_errors(V, P, alphas, s, idx, threads)
        out["fp32_vs_oracle"]["sample"] = ("%d random pairs with n <= 3000 (n <= 750 at alpha 0.75), "
                                           "oracle %.1f s" % (idx.size, time.perf_counter() - t0))
    return out


def bench_ties(dev, args, threads, do_parity):
    """Heavy-tie RNA-seq-shaped batches (negative-binomial counts, log2(c+1)):
    all 124,750 pairs of 500 variables at n=1340, and 200 pairs of 21
    variables at n=100,000 (B = 999), alpha=0.6, c=15, FP32 DP with FP64
    re-score, one gmine_compute_batch each, CUDA events around the call."""
    import torch
    from paper_1208_4271_gb300 import gmine, workloads
    out = {}
    prec = gmine.FP32_DP_FP64_RESCORE
    stream = torch.cuda.current_stream(dev)
    for key, (p, n, npairs) in (("ties_1340", (500, 1340, None)), ("ties_100000", (21, 100000, 200))):
        V, P = workloads.config5(p=p, n=n)
        if npairs is not None:
            P = P[:npairs]
        Vd = torch.from_numpy(V).to(dev)
        Pd = torch.from_numpy(np.ascontiguousarray(P)).to(dev)
        ws = gmine.Workspace(p, n, P.shape[0], ALPHA, C, prec, device=dev)
        meas = gmine.Measure(device=dev)
        gmine.compute_batch(Vd, Pd[:min(64, P.shape[0])], ALPHA, C, prec, want_M=False, workspace=ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        scores, _ = gmine.compute_batch(Vd, Pd, ALPHA, C, prec, want_M=False, workspace=ws, trace=meas.trace)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        s = gmine.scores_to_numpy(scores)
        r = {"value": P.shape[0] / (ms / 1e3), "unit": "pairs/s", "ms": ms,
             "workload": "%d pairs of %d heavy-tie variables, n=%d" % (P.shape[0], p, n),
             "dp_candidates": int(meas.counters[0].item()), "dp_ms": meas.dp_ms}
        if meas.dp_ms > 0:
            r["dp_tcand_per_s"] = r["dp_candidates"] / (meas.dp_ms / 1e3) / 1e12
        if do_parity and n <= 1340:
            rng = np.random.default_rng(55)
            idx = np.sort(rng.choice(P.shape[0], 2000, replace=False))
            t0 = time.perf_counter()
            r["fp32_vs_oracle"] = oracle_errors(V, P, ALPHA, s, idx, threads)
            r["fp32_vs_oracle"]["sample"] = "2000 random pairs, oracle %.1f s" % (time.perf_counter() - t0)
        out[key] = r
        del ws, Vd
        torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    V, P = workload(0, args.vars)
    steps = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(V, P, args.cpu_seconds / max(args.steps, 1), rng_seed=i)
        if i >= args.warmup:
            steps.append(r)
    value = statistics.mean(s["value"] for s in steps)
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(float(s["sample"].split()[0]) / s["value"] for s in steps) / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "all pairs of %d variables x n=%d (config 3), alpha=%g, c=%g"
                                   % (args.vars, N_SAMPLES, ALPHA, C)},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": steps[0]["cores"],
                             "kind": "oracle", "sample": steps[0]["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_1208_4271_gb300 import gmine, tune
    # the DP launch choices the autotuner measured on this device, if any
    # (paper_1208_4271_gb300/tuned_dp.json; the planner's rules otherwise)
    tuned_shapes = tune.apply()

    V, P = workload(rank, args.vars)
    p, n = V.shape
    npairs = P.shape[0]
    Vd = torch.from_numpy(V).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    prec = gmine.FP32_DP_FP64_RESCORE
    ws = gmine.Workspace(p, n, npairs, ALPHA, C, prec, device=dev)
    scores = torch.empty((npairs, gmine.SCORE_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    meas = gmine.Measure(device=dev)

    def step(measure=True):
        rc = gmine.lib().gmine_compute_batch_ex(
            gmine._dptr(Vd), p, n, gmine._dptr(Pd), npairs,
            gmine.ctypes.byref(gmine.Param(ALPHA, C)), prec, ws.ptr, ws.nbytes,
            gmine._dptr(scores), None, gmine.ctypes.byref(meas.trace) if measure else None,
            gmine._stream_ptr(stream))
        gmine._check(rc, "gmine_compute_batch_ex")

    for _ in range(args.warmup):
        step(measure=False)
        flush.zero_()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dp_ms = 0.0
    cand = 0
    tasks = 0
    launches = 0
    dp_launches = 0
    elapsed = 0.0
    stage_ms = dict.fromkeys(gmine.STAGE_NAMES, 0.0)
    for _ in range(args.steps):
        flush.zero_()
        e0.record(stream)
        step(measure=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        elapsed += e0.elapsed_time(e1)
        for k, v in meas.stage_ms.items():
            stage_ms[k] += v
        dp_ms += meas.dp_ms
        dp_launches += meas.dp_launches
        launches += meas.kernel_launches
        cand += int(meas.counters[0].item())
        tasks += int(meas.counters[1].item())
    barrier()
    clk = clocks.stop()
    ms_step = elapsed / args.steps
    ms_step_max = max_over_ranks(ms_step, dist, dev)
    # where a step's time goes: the call's stages (CUDA events between them,
    # summed over chunks) and the rest of the step (host work between chunks
    # that the GPU waited for, launch gaps)
    breakdown = {k: v / args.steps for k, v in stage_ms.items()}
    breakdown["outside_stages"] = ms_step - sum(breakdown.values())
    value = world * npairs / (ms_step_max / 1e3)

    # the plain FP64 DP on all pairs of the first fp64_vars variables: one
    # warm-up on a small subset, then the mean of two timed steps, each with
    # the DP launches timed by the library and their candidates counted
    fp64 = None
    if args.fp64_vars > 1:
        sub = min(args.fp64_vars, p)
        Ps = torch.from_numpy(gmine_all_pairs(sub)).to(dev)
        ws64 = gmine.Workspace(p, n, Ps.shape[0], ALPHA, C, gmine.PLAIN_FP64, device=dev)
        sc64 = torch.empty((Ps.shape[0], gmine.SCORE_DTYPE.itemsize), dtype=torch.uint8, device=dev)
        m64 = gmine.Measure(device=dev)

        def step64(npairs64, measure):
            rc = gmine.lib().gmine_compute_batch_ex(
                gmine._dptr(Vd), p, n, gmine._dptr(Ps), npairs64,
                gmine.ctypes.byref(gmine.Param(ALPHA, C)), gmine.PLAIN_FP64, ws64.ptr, ws64.nbytes,
                gmine._dptr(sc64), None, gmine.ctypes.byref(m64.trace) if measure else None,
                gmine._stream_ptr(stream))
            gmine._check(rc, "gmine_compute_batch_ex")
        step64(min(Ps.shape[0], 780), False)
        torch.cuda.synchronize(dev)
        ms64, dp64_ms, cand64, dp64_launches = 0.0, 0.0, 0, 0
        for _ in range(2):
            flush.zero_()
            e0.record(stream)
            step64(Ps.shape[0], True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms64 += e0.elapsed_time(e1) / 2
            dp64_ms += m64.dp_ms / 2
            dp64_launches += m64.dp_launches
            cand64 += int(m64.counters[0].item()) // 2
        fp64 = {"value": Ps.shape[0] / (ms64 / 1e3), "unit": "pairs/s", "ms_per_step": ms64,
                "sample": "all %d pairs of the first %d variables (%.1f %% of the workload's pairs), "
                          "mean of 2 steps after a warm-up" % (Ps.shape[0], sub, 100.0 * Ps.shape[0] / npairs),
                "dp_candidates_per_step": cand64, "dp_kernel_ms_per_step": dp64_ms,
                "dp_launches_per_step": dp64_launches // 2}
        del ws64

    # Pearson rho and the non-linearity index MIC - rho^2 of every pair of
    # the step, from the timed step's scores (inputs resident; L2 flushed
    # before each of three timed launches)
    rho_d = torch.empty(max(npairs, 1), dtype=torch.float64, device=dev)
    nl_d = torch.empty(max(npairs, 1), dtype=torch.float64, device=dev)

    def step_lin():
        rc = gmine.lib().gmine_pearson_batch(
            gmine._dptr(Vd), p, n, gmine._dptr(Pd), npairs, gmine._dptr(scores),
            gmine._dptr(rho_d), gmine._dptr(nl_d), gmine._stream_ptr(stream))
        gmine._check(rc, "gmine_pearson_batch")
    step_lin()
    torch.cuda.synchronize(dev)
    lin_ms = 0.0
    for _ in range(3):
        flush.zero_()
        e0.record(stream)
        step_lin()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        lin_ms += e0.elapsed_time(e1) / 3
    linear = {"value": world * npairs / (lin_ms / 1e3), "unit": "pairs/s", "ms": lin_ms,
              "what": "Pearson rho and MIC - rho^2 of every pair (gmine_pearson_batch, FP64), "
                      "one launch, mean of 3"}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        hv = torch.from_numpy(V).pin_memory()
        hp = torch.from_numpy(P).pin_memory()
        hs = torch.empty((npairs, gmine.SCORE_DTYPE.itemsize), dtype=torch.uint8).pin_memory()
        wsh = gmine.Workspace(p, n, npairs, ALPHA, C, prec, gmine.PLAN_HOST_STAGING, device=dev)

        def step_host():
            rc = gmine.lib().gmine_compute_batch_host(
                gmine.ctypes.c_void_p(hv.data_ptr()), p, n, gmine.ctypes.c_void_p(hp.data_ptr()),
                npairs, gmine.ctypes.byref(gmine.Param(ALPHA, C)), prec, wsh.ptr, wsh.nbytes,
                gmine.ctypes.c_void_p(hs.data_ptr()), None, gmine._stream_ptr(stream))
            gmine._check(rc, "gmine_compute_batch_host")
        step_host()
        e2e_s = 0.0
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            step_host()
            e2e_s += (time.perf_counter() - t0) / 2
        e2e = {"value": world * npairs / e2e_s, "unit": "pairs/s",
               "h2d_bytes_per_step": int(V.nbytes + P.nbytes),
               "d2h_bytes_per_step": int(npairs * gmine.SCORE_DTYPE.itemsize),
               "calls": "mean of 2 host-buffer calls after one warm-up call"}
        del wsh

    # the uneven batch and the heavy-tie batches (their own workspaces; the
    # main workload's are released first)
    del ws
    torch.cuda.empty_cache()
    threads = os.cpu_count() or 1
    do_par = rank == 0 and world == 1 and not args.no_cpu_baseline
    uneven = None if args.no_uneven else bench_uneven(dev, args, threads, do_par)
    ties = None if args.no_ties else bench_ties(dev, args, threads, do_par)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        keep = {}
        cpu = oracle_sample(V, P, args.cpu_seconds, keep=keep)
        # parity of the timed step's FP32 scores on the oracle's sample, of the
        # plain FP64 path on a sample of its subset, and the partition flips
        s32 = gmine.scores_to_numpy(scores)
        got = {k: s32[k][keep["idx"]] for k in ("mic", "mas", "mev", "mcn")}
        parity = {"fp32_vs_oracle": error_summary(got, keep["stats"]),
                  "fp32_sample_pairs": int(keep["idx"].size)}
        if fp64 is not None:
            import oracle
            s64 = gmine.scores_to_numpy(sc64)
            rng = np.random.default_rng(7)
            Ps_np = gmine_all_pairs(min(args.fp64_vars, p))
            i64 = np.sort(rng.choice(Ps_np.shape[0], min(300, Ps_np.shape[0]), replace=False))
            ref64 = oracle.score_batch(V, Ps_np[i64], ALPHA, C, nthreads=os.cpu_count() or 1)
            parity["fp64_vs_oracle"] = error_summary({k: s64[k][i64] for k in ("mic", "mas", "mev", "mcn")},
                                                     ref64["stats"])
            parity["fp64_sample_pairs"] = int(i64.size)
        parity["partition_flips_fp32"] = partition_flips(Vd, dev, min(40, p))
        # Pearson rho of the oracle's sample of pairs
        import oracle
        rho_h = rho_d.cpu().numpy()
        rerr = 0.0
        for i in keep["idx"][:2000]:
            r_ref, _ = oracle.pearson(V[P[i, 0]], V[P[i, 1]])
            if np.isnan(r_ref) != np.isnan(rho_h[i]):
                rerr = float("inf")
            elif not np.isnan(r_ref):
                rerr = max(rerr, abs(float(rho_h[i]) - r_ref))
        parity["rho_vs_oracle"] = {"max": rerr, "pairs": int(min(2000, keep["idx"].size))}

    if rank != 0:
        return
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    # ALU ceiling of the float DP: a candidate costs half a packed
    # subtraction (sub.f32x2 forms two) and half a three-operand max (one
    # merges two candidates into a running maximum): one instruction per
    # candidate on the 128 FP32 lanes of each SM at the maximum SM clock
    peak = sms * 128 * fmax * 1e6 / 1.0 / 1e12
    dp_launch_ms = dp_ms / max(dp_launches, 1)
    achieved = (cand / max(dp_launches, 1)) / (dp_launch_ms / 1e3) / 1e12 if dp_ms > 0 else 0.0
    if fp64 is not None:
        # ceiling of the double DP: one DADD per candidate on the FP64 pipe
        # (the maxima run on the integer pipe as minima of the bit patterns),
        # FP64_PER_SM_CLK of them per SM and clock
        peak64 = sms * FP64_PER_SM_CLK * fmax * 1e6 / 1.0 / 1e12
        ach64 = (fp64["dp_candidates_per_step"] / (fp64["dp_kernel_ms_per_step"] / 1e3) / 1e12
                 if fp64["dp_kernel_ms_per_step"] > 0 else 0.0)
        fp64["roofline"] = {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "Tcand/s",
                            "frac": ach64 / peak64,
                            "peak_basis": "%d SMs x %d FP64 ops/clk x %.0f MHz / 1 FP64 op per DP step "
                                          "(DADD; the max on the integer pipe)" % (sms, FP64_PER_SM_CLK, fmax)}
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "all pairs of %d variables x n=%d (config 3: log-normal "
                                   "expression, 40 co-regulated modules), alpha=%g, c=%g"
                                   % (p, n, ALPHA, C),
                       "pairs_per_gpu": npairs, "dp": "fp32 with int32 counts, fp64 re-score",
                       "dp_plan": ("autotuned (%d cached shapes of this device applied)" % tuned_shapes
                                   if tuned_shapes else "planner rules"),
                       "l2": "256 MiB buffer written between timed steps"},
            "plain_fp64": fp64,
            "linear": linear,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tcand/s",
                         "frac": achieved / peak if peak else None,
                         "traffic": DP_DRAM_BYTES_PER_TASK * (tasks / max(args.steps, 1))
                                    / max(dp_launches // max(args.steps, 1), 1),
                         "traffic_basis": "bytes per average DP launch: %.1f KB per task (ncu, 60-variable "
                                          "launch list) x tasks per step / DP launches per step"
                                          % (DP_DRAM_BYTES_PER_TASK / 1e3),
                         "kernel": "OptimizeXAxis DP launches (k_dp, k_dp_warp, k_dp_mid, k_dp_small, k_dp_two)",
                         "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz / 1 instr per DP step "
                                       "(half a packed sub.f32x2 + half a 3-operand max)" % (sms, fmax),
                         "dp_candidates_per_step": cand // max(args.steps, 1),
                         "dp_kernel_ms_per_step": dp_ms / args.steps,
                         "dp_launches_per_step": dp_launches // args.steps,
                         "tasks_per_step": tasks // args.steps},
            "step_breakdown_ms": breakdown,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "parity": parity,
            "uneven": uneven,
            "ties": ties}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def gmine_all_pairs(p):
    from paper_1208_4271_gb300 import workloads
    return workloads.all_pairs(p)


if __name__ == "__main__":
    main()
