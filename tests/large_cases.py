"""Inputs and oracle results of the largest parity cases (tests/test_gpu_large.py).

The oracle needs minutes for these (one pair at n = 100,000 runs the DP over
thousands of superclumps for hundreds of row counts on one core), so its
results are computed in a background thread that starts when the session has
collected the tests that use them; the GPU tests before them run meanwhile.
Each oracle call is a ctypes call that releases the GIL, one pair or task per
worker thread.

Cases:
  n100k  n = 100,000, alpha = 0.6 (B = 999, 5,056 cells): a heavy-tie pair
         from the negative-binomial count generator (log2(count + 1)), a
         continuous pair with small noise, and a noiseless monotone pair;
  a075   alpha = 0.75: a rounded pair at n = 20,000 (B = 1,681; about 2,000
         distinct values per variable) and uneven pairs with missing samples
         from the uneven-batch generator, n up to 6,000.
"""
import queue
import threading

import numpy as np

C = 15.0
TASKS_N100K = [(0, o, y) for o in (0, 1) for y in (2, 3, 40, 300, 499)]

_lock = threading.Lock()
_jobs = None
_futures = {}


class _Job:
    """A call run by a daemon worker thread (a run stopped early does not
    wait for the oracle at exit)."""

    def __init__(self, fn, *args):
        self.fn, self.args = fn, args
        self.done = threading.Event()
        self.value = self.error = None

    def run(self):
        try:
            self.value = self.fn(*self.args)
        except BaseException as e:  # handed to the test that waits for it
            self.error = e
        self.done.set()

    def result(self):
        self.done.wait()
        if self.error is not None:
            raise self.error
        return self.value


def _worker():
    while True:
        _jobs.get().run()


def _submit(fn, *args):
    j = _Job(fn, *args)
    _jobs.put(j)
    return j


def n100k():
    from paper_1208_4271_gb300 import workloads
    n = 100000
    Vnb, _ = workloads.config5(p=2, n=n, seed_salt=100)
    rng = np.random.default_rng(100000)
    x = rng.random(n)
    V = np.empty((6, n))
    V[0], V[1] = Vnb[0], Vnb[1]
    V[2] = x
    V[3] = x + 0.01 * rng.standard_normal(n)
    V[4] = rng.random(n)
    V[5] = np.exp(3.0 * V[4])
    P = np.array([[0, 1], [2, 3], [4, 5]], dtype=np.int32)
    return V, P, 0.6


def a075():
    from paper_1208_4271_gb300 import workloads
    n = 20000
    rng = np.random.default_rng(75)
    Vu, Pu, _, _ = workloads.config4(n_pairs=12, n_lo=1000, n_hi=6000, seed_salt=75)
    V = np.full((2 + Vu.shape[0], n), np.nan)
    x = np.round(rng.random(n) * 2000.0)
    V[0] = x
    V[1] = np.round(x + 300.0 * rng.standard_normal(n))
    V[2:, :Vu.shape[1]] = Vu
    P = np.concatenate([np.array([[0, 1]], dtype=np.int32), Pu + 2]).astype(np.int32)
    return V, P, 0.75


CASES = {"n100k": n100k, "a075": a075}


def _pair_job(V, P, i, alpha):
    import oracle
    return oracle.score_batch(V, P[i:i + 1], alpha, C, nthreads=1, want_M=True)


def _task_job(V, P, i, o, y, alpha):
    from gpu_util import oracle_task
    return oracle_task(V, P, i, o, y, alpha, C)


def start(workers=24):
    """Start every oracle job of every case (idempotent)."""
    global _jobs
    with _lock:
        if _jobs is not None:
            return
        _jobs = queue.Queue()
        for _ in range(workers):
            threading.Thread(target=_worker, daemon=True).start()
        for name, make in CASES.items():
            V, P, alpha = make()
            _futures[name] = {"input": (V, P, alpha),
                              "pairs": [_submit(_pair_job, V, P, i, alpha) for i in range(P.shape[0])]}
        V, P, alpha = _futures["n100k"]["input"]
        _futures["n100k"]["tasks"] = {t: _submit(_task_job, V, P, t[0], t[1], t[2], alpha)
                                      for t in TASKS_N100K}


def case(name):
    """(V, P, alpha) of a case."""
    start()
    return _futures[name]["input"]


def oracle_pairs(name):
    """The oracle's score_batch result for every pair of a case, merged."""
    start()
    parts = [f.result() for f in _futures[name]["pairs"]]
    out = {"stats": np.concatenate([p["stats"] for p in parts]),
           "info": np.concatenate([p["info"] for p in parts]),
           "status": np.concatenate([p["status"] for p in parts])}
    Ms, offs, o = [], [], 0
    for p in parts:
        offs.append(o)
        Ms.append(p["M"][:int(p["info"][0, 3])])
        o += Ms[-1].size
    out["M"] = np.concatenate(Ms) if Ms else np.zeros(1)
    out["M_offsets"] = np.array(offs, dtype=np.int64)
    return out


def oracle_tasks(name):
    start()
    return {t: f.result() for t, f in _futures[name]["tasks"].items()}
