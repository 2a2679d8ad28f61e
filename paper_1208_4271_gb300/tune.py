"""Autotuner of the OptimizeXAxis launch plan.

For a batch shape (n samples, alpha, c, precision) the planner splits the
row counts y into launch groups and gives each a kernel shape (blocked CTA
per task, warp per task, level-major, small, two-column) and a CTA size by
fixed rules.  The tuner measures instead: on a synthetic sample of the
shape (all pairs of a few variables of the microarray-shaped generator, one
chunk), for each launch group in turn it times every kernel shape and CTA
size the library accepts for that group (gmine_set_dp_choices, then the
per-launch CUDA-event times of gmine_trace), keeps a candidate only if its
scores equal those of the built-in plan (bit for bit on the plain FP64 path,
within 1e-9 on the float path, whose re-score order differs between
shapes), and keeps the fastest.  The choices are cached in a JSON file keyed
by device and shape; apply() hands the cached choices of the current device
to the library, which uses them for calls planned afterwards and keeps its
rules wherever a choice does not fit.

    python -m paper_1208_4271_gb300.tune --n 1340 --alpha 0.6 --precision 1
"""
import argparse
import json
import os

import numpy as np

from . import gmine

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuned_dp.json")


def cache_path():
    return os.environ.get("GMINE_TUNE_CACHE", DEFAULT_CACHE)


def candidates(group, B, fp32):
    """Kernel shapes and CTA sizes to try for a launch group (the library
    decides which of them apply to the group)."""
    x_lo = B // group["ylo"]
    out = []
    if x_lo == 2:
        out += [(gmine.DP_TWO, t) for t in (64, 128, 256)]
    out += [(gmine.DP_BLOCKED, t) for t in (128, 256)]
    if fp32 and group["yhi"] <= 15:
        out += [(gmine.DP_WARP, t) for t in (32, 64, 128, 224)]
    out += [(gmine.DP_MID, t) for t in (128, 256)]
    if x_lo <= 9:
        out += [(gmine.DP_SMALL, t) for t in (32, 64, 128)]
    return out


def same_scores(a, b, exact):
    if not np.array_equal(a["status"], b["status"]):
        return False
    for k in ("mic", "mas", "mev"):
        if exact and not np.array_equal(a[k], b[k]):
            return False
        if not exact and np.max(np.abs(a[k] - b[k]), initial=0.0) > 1e-9:
            return False
    return True


class GpuBackend:
    """Runs the sample batch on the current GPU through the C ABI."""

    def __init__(self, n, alpha, c, precision, n_vars=60, reps=2, device="cuda"):
        import torch
        from . import workloads
        self.shape = (n, alpha, c, precision)
        V, P = workloads.config3(p=n_vars, n=n)
        self.Vd = torch.from_numpy(V).to(device)
        self.Pd = torch.from_numpy(P).to(device)
        self.reps = reps
        self.device = device
        self.device_name = torch.cuda.get_device_name(torch.device(device))

    def set_choices(self, choices):
        n, alpha, c, precision = self.shape
        gmine.set_dp_choices(n, alpha, c, precision, choices)

    def groups(self):
        n, alpha, c, precision = self.shape
        return gmine.dp_groups(n, alpha, c, precision)

    def run(self):
        """(per-group milliseconds, median over reps; scores)."""
        import torch
        n, alpha, c, precision = self.shape
        m = gmine.Measure(device=self.device)
        # planned under the choices now set (they may need another workspace)
        ws = gmine.Workspace(self.Vd.shape[0], n, self.Pd.shape[0], alpha, c, precision,
                             device=self.device)
        times = []
        for _ in range(self.reps):
            sc, _ = gmine.compute_batch(self.Vd, self.Pd, alpha, c, precision, want_M=False,
                                        workspace=ws, trace=m.trace)
            torch.cuda.synchronize()
            times.append(m.launch_ms)
        return np.median(np.stack(times), axis=0), gmine.scores_to_numpy(sc)


def tune(backend, log=None):
    """Choose each launch group's kernel shape and CTA size by measurement.
    Returns the cache entry {device, n, alpha, c, precision, groups: [...]}
    and leaves the chosen set active in the library."""
    n, alpha, c, precision = backend.shape
    fp32 = precision == gmine.FP32_DP_FP64_RESCORE
    B = gmine.B_of(n, alpha)
    backend.set_choices([])
    default = backend.groups()
    base_ms, ref = backend.run()
    chosen = []
    rows = []
    for gi, g in enumerate(default):
        best = {"ylo": g["ylo"], "yhi": g["yhi"], "kind": g["kind"], "threads": g["threads"]}
        best_ms = float(base_ms[gi])
        tried = []
        for kind, threads in candidates(g, B, fp32):
            cand = {"ylo": g["ylo"], "yhi": g["yhi"], "kind": kind, "threads": threads}
            backend.set_choices(chosen + [cand])
            eff = backend.groups()
            if len(eff) != len(default) or eff[gi]["kind"] != kind or eff[gi]["threads"] != threads:
                continue  # does not apply to this group, or does not fit
            ms, scores = backend.run()
            if not same_scores(scores, ref, exact=not fp32):
                tried.append((kind, threads, None))
                continue
            tried.append((kind, threads, float(ms[gi])))
            if ms[gi] < best_ms:
                best_ms = float(ms[gi])
                best = cand
        chosen.append(best)
        rows.append(dict(best, ms=best_ms, default_kind=g["kind"], default_threads=g["threads"],
                         default_ms=float(base_ms[gi]), tried=tried))
        if log:
            log("group y=%d..%d: %s/%d %.4f ms (rules: %s/%d %.4f ms)" % (
                g["ylo"], g["yhi"], gmine.DP_KIND_NAMES[best["kind"]], best["threads"], best_ms,
                gmine.DP_KIND_NAMES[g["kind"]], g["threads"], float(base_ms[gi])))
    backend.set_choices(chosen)
    return {"device": backend.device_name, "n": int(n), "alpha": float(alpha), "c": float(c),
            "precision": int(precision), "groups": rows}


def _key(e):
    return (e["device"], e["n"], e["alpha"], e["c"], e["precision"])


def load(path=None):
    path = path or cache_path()
    if not os.path.exists(path):
        return []
    with open(path) as f:
        return json.load(f)


def save(entry, path=None):
    """Merge an entry into the cache file (an entry of the same device and
    shape is replaced)."""
    path = path or cache_path()
    entries = [e for e in load(path) if _key(e) != _key(entry)]
    entries.append(entry)
    entries.sort(key=_key)
    with open(path + ".tmp", "w") as f:
        json.dump(entries, f, indent=1)
    os.replace(path + ".tmp", path)


def apply(entries=None, device_name=None, setter=None):
    """Hand the cached choices of this device to the library; returns how
    many shapes were applied.  A group whose measured best was the planner's
    own choice at tuning time is left to the planner's rules (which may have
    improved since); only the choices that beat the rules are handed over."""
    if entries is None:
        entries = load()
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    setter = setter or gmine.set_dp_choices
    k = 0
    for e in entries:
        if e["device"] != device_name:
            continue
        setter(e["n"], e["alpha"], e["c"], e["precision"],
               [{f: g[f] for f in ("ylo", "yhi", "kind", "threads")} for g in e["groups"]
                if (g["kind"], g["threads"]) != (g.get("default_kind"), g.get("default_threads"))])
        k += 1
    return k


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=1340)
    ap.add_argument("--alpha", type=float, default=0.6)
    ap.add_argument("--c", type=float, default=15.0)
    ap.add_argument("--precision", type=int, default=gmine.FP32_DP_FP64_RESCORE)
    ap.add_argument("--vars", type=int, default=60)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    be = GpuBackend(a.n, a.alpha, a.c, a.precision, a.vars, a.reps)
    entry = tune(be, log=print)
    save(entry, a.out)
    print("saved", a.out or cache_path())


if __name__ == "__main__":
    main()
