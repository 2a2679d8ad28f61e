"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no MINE arithmetic: it only draws variables.  Both the CUDA
path and the CPU oracle are fed from here.  The paper's datasets (Spellman,
microbiome, GSE25219, GSE34914) are not available, so every workload is a
synthetic stand-in with the shape the paper reports (Table 1; SI Sec. 2C, 3A,
3B) and the value structure described in each function.

Layout: a variable matrix ``vars`` of shape [p, n], float64, one variable per
row (the paper's files are variables by samples), NaN for a missing sample,
and a pair list ``pairs`` of shape [n_pairs, 2], int32.
"""
import numpy as np

SEED0 = 20120822


def _rng(config_id, salt=0):
    return np.random.default_rng(SEED0 + 1000 * salt + config_id)


def all_pairs(p):
    """All unordered pairs (i, j), i < j, in row-major order."""
    iu, ju = np.triu_indices(p, k=1)
    return np.stack([iu, ju], axis=1).astype(np.int32)


def cpp_example():
    """The C++ example of the paper (Sec. Examples): n = 1001 points,
    x_i = i/1000, y = sin(10*PI*x) + x with PI = 3.14159265."""
    n = 1001
    PI = 3.14159265
    x = np.arange(n, dtype=np.float64) / float(n - 1)
    y = np.sin(10.0 * PI * x) + x
    return np.stack([x, y]), np.array([[0, 1]], dtype=np.int32)


def config1(seed_salt=0):
    """16 pairs, n = 300: x ~ U(0,1); y = x, 4x(1-x), sin(8 pi x) and an
    independent U(0,1), each clean and with N(0, 0.1^2) noise; 8 kinds x 2
    draws.  Returns (vars [32, 300], pairs [16, 2])."""
    rng = _rng(1, seed_salt)
    n = 300
    rows = []
    for draw in range(2):
        for noisy in (False, True):
            for kind in range(4):
                x = rng.uniform(0.0, 1.0, n)
                if kind == 0:
                    y = x.copy()
                elif kind == 1:
                    y = 4.0 * x * (1.0 - x)
                elif kind == 2:
                    y = np.sin(8.0 * np.pi * x)
                else:
                    y = rng.uniform(0.0, 1.0, n)
                if noisy:
                    y = y + rng.normal(0.0, 0.1, n)
                rows.append(x)
                rows.append(y)
    vars_ = np.stack(rows)
    pairs = np.arange(vars_.shape[0], dtype=np.int32).reshape(-1, 2)
    return vars_, pairs


def config2(seed_salt=0):
    """100 variables x n = 1000, all 4950 pairs: 50 iid N(0,1) and 50 noisy
    functions (linear, quadratic, exponential, sinusoid of frequency 1-8,
    circle) of a randomly chosen earlier variable, noise sd ~ U(0,1)."""
    rng = _rng(2, seed_salt)
    n = 1000
    p = 100
    V = np.empty((p, n))
    V[:50] = rng.normal(0.0, 1.0, (50, n))
    for i in range(50, p):
        u = V[rng.integers(0, i)]
        kind = int(rng.integers(0, 5))
        sd = rng.uniform(0.0, 1.0)
        if kind == 0:
            y = 2.0 * u + 1.0
        elif kind == 1:
            y = u * u
        elif kind == 2:
            y = np.exp(np.clip(u, -20, 20))
        elif kind == 3:
            f = rng.uniform(1.0, 8.0)
            y = np.sin(2.0 * np.pi * f * u)
        else:
            s = 2.0 * (u - u.min()) / max(u.max() - u.min(), 1e-300) - 1.0
            sign = rng.choice([-1.0, 1.0], n)
            y = sign * np.sqrt(np.clip(1.0 - s * s, 0.0, None))
        V[i] = y + rng.normal(0.0, sd, n) * max(np.std(y), 1e-12)
    return V, all_pairs(p)


def config3(p=2000, n=1340, seed_salt=0):
    """Microarray-shaped matrix (stands in for GSE25219, n = 1340): p genes in
    modules of 50 sharing a latent factor f, z = lam*f + sqrt(1-lam^2)*eps
    with lam ~ U(0.3, 0.9); 10 % of the genes instead follow a monotone
    (exp / cubic) or sinusoidal function of f; expression = exp(6 + 1.5 z).
    All p(p-1)/2 pairs."""
    rng = _rng(3, seed_salt)
    mod_size = 50
    n_mod = (p + mod_size - 1) // mod_size
    F = rng.normal(0.0, 1.0, (n_mod, n))
    V = np.empty((p, n))
    for g in range(p):
        f = F[g // mod_size]
        lam = rng.uniform(0.3, 0.9)
        eps = rng.normal(0.0, 1.0, n)
        if rng.uniform() < 0.10:
            kind = int(rng.integers(0, 3))
            if kind == 0:
                h = np.exp(0.8 * f)
            elif kind == 1:
                h = f ** 3
            else:
                h = np.sin(2.0 * f)
            h = (h - h.mean()) / max(h.std(), 1e-12)
            z = lam * h + np.sqrt(1.0 - lam * lam) * eps
        else:
            z = lam * f + np.sqrt(1.0 - lam * lam) * eps
        V[g] = np.exp(6.0 + 1.5 * z)
    return V, all_pairs(p)


def config4(n_pairs=20000, n_lo=50, n_hi=20000, seed_salt=0):
    """Uneven batch: n_pairs independent pairs, n log-uniform in [n_lo, n_hi],
    0-20 % of the samples of each pair set to NaN, relationship drawn from
    {independent, linear, parabolic, sinusoid, step, circle} with noise sd in
    [0, 1], alpha drawn from {0.55, 0.6, 0.75}.  Pairs are padded with NaN to
    the longest n.  Returns (vars [2*n_pairs, n_max], pairs, alpha per pair,
    n per pair)."""
    rng = _rng(4, seed_salt)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), n_pairs)).astype(np.int64)
    nmax = int(ns.max())
    V = np.full((2 * n_pairs, nmax), np.nan)
    alphas = rng.choice(np.array([0.55, 0.6, 0.75]), n_pairs)
    for i in range(n_pairs):
        n = int(ns[i])
        x = rng.uniform(-1.0, 1.0, n)
        kind = int(rng.integers(0, 6))
        sd = rng.uniform(0.0, 1.0)
        if kind == 0:
            y = rng.uniform(-1.0, 1.0, n)
        elif kind == 1:
            y = x.copy()
        elif kind == 2:
            y = x * x
        elif kind == 3:
            y = np.sin(2.0 * np.pi * rng.uniform(1.0, 4.0) * x)
        elif kind == 4:
            y = np.where(x > rng.uniform(-0.5, 0.5), 1.0, 0.0)
        else:
            y = np.sign(rng.uniform(-1, 1, n)) * np.sqrt(np.clip(1.0 - x * x, 0.0, None))
        y = y + rng.normal(0.0, sd, n) * 0.5
        frac = rng.uniform(0.0, 0.2)
        miss_x = rng.uniform(0, 1, n) < frac / 2
        miss_y = rng.uniform(0, 1, n) < frac / 2
        x[miss_x] = np.nan
        y[miss_y] = np.nan
        V[2 * i, :n] = x
        V[2 * i + 1, :n] = y
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return V, pairs, alphas, ns


def config5(p=500, n=1340, seed_salt=0):
    """RNA-seq-shaped counts with heavy ties (stands in for GSE34914-like
    data): negative binomial counts with mean log-uniform in [1, 1000] and
    dispersion in [0.1, 2], transformed to log2(count + 1).  All pairs."""
    rng = _rng(5, seed_salt)
    mu = np.exp(rng.uniform(0.0, np.log(1000.0), p))
    disp = rng.uniform(0.1, 2.0, p)
    F = rng.normal(0.0, 1.0, ((p + 49) // 50, n))
    V = np.empty((p, n))
    for g in range(p):
        lam = rng.uniform(0.0, 0.8)
        z = lam * F[g // 50] + np.sqrt(1 - lam * lam) * rng.normal(0.0, 1.0, n)
        m = mu[g] * np.exp(0.5 * z)
        r = 1.0 / disp[g]
        prob = r / (r + m)
        counts = rng.negative_binomial(r, prob)
        V[g] = np.log2(counts + 1.0)
    return V, all_pairs(p)


def tie_heavy(p=8, n=400, levels=6, seed_salt=0):
    """Small integer-valued variables (few distinct values): exercises tie
    groups in EquipartitionYAxis and mixed x-tie runs in GetClumpsPartition."""
    rng = _rng(6, seed_salt)
    V = rng.integers(0, levels, (p, n)).astype(np.float64)
    V[1::2] = V[0::2] + rng.integers(0, 2, (p // 2, n))
    return V, all_pairs(p)


def uniform_pairs(n, reps, seed_salt=0):
    """The scaling experiment's input (SI Sec. 2C): reps independent pairs of
    two uniformly distributed random vectors of length n (the paper times
    100 replicates per size).  Returns (vars [2*reps, n], pairs [reps, 2])."""
    rng = _rng(7, 1000 * seed_salt + int(n))
    V = rng.uniform(0.0, 1.0, (2 * reps, n))
    pairs = np.arange(2 * reps, dtype=np.int32).reshape(-1, 2)
    return V, pairs


def sparse_count_pairs(n=675, n_pairs=6, seed_salt=0):
    """Stand-in for the microbiome OTU pairs of the c-convergence figure
    (SI Sec. 1, n = 675 samples, alpha = 0.551): sparse abundance counts with
    many zeros (heavy ties), each pair sharing a latent factor through a
    different relation (monotone, quadratic, threshold), so that clumps and
    superclumps matter.  Returns (vars [2*n_pairs, n], pairs)."""
    rng = _rng(8, seed_salt)
    V = np.empty((2 * n_pairs, n))
    for i in range(n_pairs):
        f = rng.normal(0.0, 1.0, n)
        kind = i % 3
        if kind == 0:
            g = f + 0.5 * rng.normal(0.0, 1.0, n)
        elif kind == 1:
            g = f * f - 1.0 + 0.5 * rng.normal(0.0, 1.0, n)
        else:
            g = np.where(f > 0.3, 1.5, -0.5) + 0.5 * rng.normal(0.0, 1.0, n)
        for j, z in enumerate((f, g)):
            present = rng.uniform(0.0, 1.0, n) < rng.uniform(0.3, 0.7)  # many absent taxa
            mean = np.exp(1.5 + 0.8 * z)
            V[2 * i + j] = np.where(present, rng.poisson(mean), 0).astype(np.float64)
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return V, pairs
