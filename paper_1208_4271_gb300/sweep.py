"""Parameter sweeps of the batched MINE path on synthetic stand-ins.

time  -- the scaling experiment (SI Sec. 2C): two uniformly distributed
         random vectors of length n, for several n and alpha; the paper times
         100 replicates of one pair per size on a laptop.  Here the
         replicates of one (n, alpha) form one batch on the GPU, timed with
         CUDA events after a warm-up, in each precision; per size the time
         ratio of alpha = 0.6 to alpha = 0.7 is reported too (the paper finds
         the former below 15 % of the latter).
c     -- convergence in c (the c-sweep figure of SI Sec. 1): MIC of sparse
         abundance-count pairs (n = 675, alpha = 0.551, as the microbiome
         analysis) for increasing c, and each value's distance to the MIC at
         the largest c: the superclump step merges fewer clumps as c grows.

One JSON line per measurement on stdout.  --dry-run prints the plan without
touching a GPU.  Usage:
    python -m paper_1208_4271_gb300.sweep time --sizes 250,500,1000 --alphas 0.5,0.6,0.7
    python -m paper_1208_4271_gb300.sweep c --cs 1,2,5,10,15,30,60,120
"""
import argparse
import json
import sys

import numpy as np

from . import workloads

PRECISIONS = {"fp64": 0, "fp32": 1}


def _floats(text):
    return [float(v) for v in text.split(",") if v]


def _ints(text):
    return [int(v) for v in text.split(",") if v]


def time_plan(sizes, alphas, precisions):
    return [{"sweep": "time", "n": n, "alpha": a, "precision": p}
            for n in sizes for a in alphas for p in precisions]


def c_plan(cs, precisions):
    return [{"sweep": "c", "c": c, "precision": p} for c in cs for p in precisions]


def time_sweep(sizes, alphas, reps=100, c=15.0, precisions=("fp32", "fp64"), repeats=3, seed_salt=0):
    """Records {n, alpha, precision, pairs, ms_per_pair, pairs_per_s} for
    every (n, alpha, precision), then {n, precision, ratio_06_07} where both
    alphas were timed."""
    import torch
    from . import gmine
    dev = torch.device("cuda", torch.cuda.current_device())
    out = []
    for n in sizes:
        V, P = workloads.uniform_pairs(n, reps, seed_salt)
        Vd = torch.from_numpy(V).to(dev)
        Pd = torch.from_numpy(P).to(dev)
        for prec in precisions:
            code = PRECISIONS[prec]
            for a in alphas:
                ws = gmine.Workspace(V.shape[0], n, reps, a, c, code, device=dev)
                gmine.compute_batch(Vd, Pd, a, c, code, want_M=False, workspace=ws)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                ms = 0.0
                for _ in range(repeats):
                    e0.record()
                    gmine.compute_batch(Vd, Pd, a, c, code, want_M=False, workspace=ws)
                    e1.record()
                    torch.cuda.synchronize(dev)
                    ms += e0.elapsed_time(e1) / repeats
                out.append({"sweep": "time", "n": n, "alpha": a, "c": c, "precision": prec,
                            "pairs": reps, "ms_per_batch": ms, "ms_per_pair": ms / reps,
                            "pairs_per_s": reps / (ms / 1e3)})
                del ws
            t = {r["alpha"]: r["ms_per_batch"] for r in out
                 if r["sweep"] == "time" and r["n"] == n and r["precision"] == prec}
            if 0.6 in t and 0.7 in t:
                out.append({"sweep": "time_ratio", "n": n, "precision": prec,
                            "ratio_06_07": t[0.6] / t[0.7]})
    return out


def c_sweep(cs, n=675, n_pairs=6, alpha=0.551, precisions=("fp64", "fp32"), seed_salt=0):
    """Records {c, precision, mic (per pair)} for every c, then per
    precision the distance of each c's MIC to the largest c's."""
    import torch
    from . import gmine
    dev = torch.device("cuda", torch.cuda.current_device())
    V, P = workloads.sparse_count_pairs(n, n_pairs, seed_salt)
    Vd = torch.from_numpy(V).to(dev)
    Pd = torch.from_numpy(P).to(dev)
    out = []
    for prec in precisions:
        mics = {}
        for c in cs:
            scores, _ = gmine.compute_batch(Vd, Pd, alpha, c, PRECISIONS[prec], want_M=False)
            torch.cuda.synchronize(dev)
            mics[c] = gmine.scores_to_numpy(scores)["mic"].astype(np.float64)
            out.append({"sweep": "c", "c": c, "alpha": alpha, "n": n, "precision": prec,
                        "mic": mics[c].tolist()})
        cmax = max(cs)
        for c in cs:
            out.append({"sweep": "c_convergence", "c": c, "c_max": cmax, "precision": prec,
                        "max_abs_diff_to_c_max": float(np.max(np.abs(mics[c] - mics[cmax])))})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("mode", choices=["time", "c"])
    ap.add_argument("--sizes", default="250,500,1000,2000,4000")
    ap.add_argument("--alphas", default="0.5,0.6,0.7")
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--cs", default="1,2,5,10,15,20,30,60,120")
    ap.add_argument("--n", type=int, default=675)
    ap.add_argument("--pairs", type=int, default=6)
    ap.add_argument("--alpha", type=float, default=0.551)
    ap.add_argument("--c", type=float, default=15.0)
    ap.add_argument("--precision", choices=["fp32", "fp64", "both"], default="both")
    ap.add_argument("--dry-run", action="store_true")
    args = ap.parse_args(argv)
    precs = ["fp32", "fp64"] if args.precision == "both" else [args.precision]
    if args.mode == "time":
        sizes, alphas = _ints(args.sizes), _floats(args.alphas)
        recs = (time_plan(sizes, alphas, precs) if args.dry_run
                else time_sweep(sizes, alphas, args.reps, args.c, precs))
    else:
        cs = _floats(args.cs)
        recs = (c_plan(cs, precs) if args.dry_run
                else c_sweep(cs, args.n, args.pairs, args.alpha, precs))
    for r in recs:
        print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
