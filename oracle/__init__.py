"""ctypes wrapper around the FP64 CPU oracle (oracle/mine_oracle.c).

Test infrastructure only.  The product path (the CUDA library and its Python
binding) never imports this package; only tests/, the smoke check and the
CPU-baseline leg of bench.py do.

Each wrapper names the step of the method it exposes; the C file carries the
citations and the readings of the paper.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

STATUS = {0: "OK", 1: "E_PARAM", 2: "E_TOO_FEW", 3: "E_CONSTANT", 4: "E_NOMEM"}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_B.argtypes = [ctypes.c_int, ctypes.c_double]
        L.oracle_B.restype = ctypes.c_int
        L.oracle_khat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.oracle_khat.restype = ctypes.c_int
        L.oracle_m_cells.argtypes = [ctypes.c_int]
        L.oracle_m_cells.restype = ctypes.c_int
        L.oracle_argsort.argtypes = [_dp, ctypes.c_int, _ip]
        L.oracle_argsort.restype = ctypes.c_int
        L.oracle_equipartition.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip]
        L.oracle_equipartition.restype = ctypes.c_int
        L.oracle_clumps.argtypes = [_dp, _ip, ctypes.c_int, _ip]
        L.oracle_clumps.restype = ctypes.c_int
        L.oracle_superclumps.argtypes = [_dp, _ip, ctypes.c_int, ctypes.c_int, _ip]
        L.oracle_superclumps.restype = ctypes.c_int
        L.oracle_optimize_x_axis.argtypes = [_dp, _ip, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, _dp, _ip,
                                             _ip, _ip, ctypes.c_int]
        L.oracle_optimize_x_axis.restype = ctypes.c_int
        L.oracle_check_param.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_check_param.restype = ctypes.c_int
        L.oracle_score_pair.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _dp, _dp, _ip]
        L.oracle_score_pair.restype = ctypes.c_int
        L.oracle_score_batch.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip,
                                         ctypes.c_long, ctypes.c_double,
                                         ctypes.c_double, _dp, _ip, _ip, _dp,
                                         _lp, ctypes.c_int]
        L.oracle_score_batch.restype = ctypes.c_int
        L.oracle_score_batch_alphas.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip,
                                                ctypes.c_long, _dp, ctypes.c_double, _dp, _ip,
                                                _ip, _dp, _lp, ctypes.c_int]
        L.oracle_score_batch_alphas.restype = ctypes.c_int
        L.oracle_pearson.argtypes = [_dp, _dp, ctypes.c_int, _ip]
        L.oracle_pearson.restype = ctypes.c_double
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


def B_of(n, alpha):
    """B = floor(n^alpha) (Sec. 2C)."""
    return lib().oracle_B(int(n), float(alpha))


def khat_of(B, y, c):
    """khat = max(floor(c * floor(B/y)), 1) (Appendix item 7)."""
    return lib().oracle_khat(int(B), int(y), float(c))


def m_cells(B):
    """Number of cells (x, y), x, y >= 2, xy <= B."""
    return lib().oracle_m_cells(int(B))


def cell_layout(B):
    """The (x, y) of each stored cell of M, y-major then x."""
    return [(x, y) for y in range(2, B // 2 + 1) for x in range(2, B // y + 1)]


def argsort(v):
    v = _d(v)
    out = np.empty(len(v), dtype=np.int32)
    lib().oracle_argsort(_pd(v), len(v), _pi(out))
    return out


def equipartition(v, y):
    """EquipartitionYAxis (SOM Alg. 3): returns (Q per sample, yhat)."""
    v = _d(v)
    Q = np.empty(len(v), dtype=np.int32)
    yhat = lib().oracle_equipartition(_pd(v), len(v), int(y), _pi(Q))
    return Q, yhat


def clumps(u, Q):
    """GetClumpsPartition: returns (clump per sample, k)."""
    u, Q = _d(u), _i(Q)
    P = np.empty(len(u), dtype=np.int32)
    k = lib().oracle_clumps(_pd(u), _pi(Q), len(u), _pi(P))
    return P, k


def superclumps(u, Q, khat):
    """GetSuperclumpsPartition: returns (superclump per sample, k)."""
    u, Q = _d(u), _i(Q)
    P = np.empty(len(u), dtype=np.int32)
    k = lib().oracle_superclumps(_pd(u), _pi(Q), len(u), int(khat), _pi(P))
    return P, k


def optimize_x_axis(u, Q, yhat, x, khat):
    """OptimizeXAxis: returns dict(I[l-2], cuts[l-2] (list), k, sc_ends)."""
    u, Q = _d(u), _i(Q)
    n = len(u)
    I = np.empty(max(x - 1, 0), dtype=np.float64)
    cuts = np.empty(max(x * (x - 1) // 2, 1), dtype=np.int32)
    k = ctypes.c_int(0)
    ends = np.empty(n + 1, dtype=np.int32)
    rc = lib().oracle_optimize_x_axis(_pd(u), _pi(Q), n, int(yhat), int(x), int(khat),
                                      _pd(I), _pi(cuts), ctypes.byref(k), _pi(ends), n + 1)
    if rc != 0:
        raise RuntimeError("oracle_optimize_x_axis: " + STATUS.get(rc, str(rc)))
    kk = k.value
    cl = []
    for l in range(2, x + 1):
        off = (l - 2) * (l - 1) // 2
        cl.append(cuts[off:off + l - 1].tolist())
    return {"I": I, "cuts": cl, "k": kk, "sc_ends": ends[:kk + 1].copy()}


def score_pair(x, y, alpha=0.6, c=15.0):
    """mine_compute_score for one pair: M, MIC, MAS, MEV, MCN and bookkeeping."""
    x, y = _d(x), _d(y)
    n = len(x)
    assert len(y) == n
    n_used = int(np.count_nonzero(np.isfinite(x) & np.isfinite(y)))
    cells = max(m_cells(B_of(max(n_used, 1), alpha)), 1)
    M = np.zeros(cells, dtype=np.float64)
    stats = np.zeros(4, dtype=np.float64)
    info = np.zeros(6, dtype=np.int32)
    st = lib().oracle_score_pair(_pd(x), _pd(y), n, float(alpha), float(c),
                                 _pd(M), _pd(stats), _pi(info))
    return {"status": int(st), "mic": stats[0], "mas": stats[1], "mev": stats[2],
            "mcn": stats[3], "n_used": int(info[0]), "B": int(info[1]),
            "mcn_xy": int(info[2]), "m_cells": int(info[3]),
            "yhat0": int(info[4]), "yhat1": int(info[5]),
            "M": M[:int(info[3])].copy()}


def score_batch(vars_, pairs, alpha=0.6, c=15.0, nthreads=0, want_M=False):
    """All listed pairs of the rows of vars_ ([p, n]); OpenMP over pairs.
    alpha: one value, or one per pair (B = n^alpha of each pair, Sec. 2C).

    Returns dict(stats [npairs, 4], info [npairs, 6], status [npairs],
    M (concatenated cells) and M_offsets when want_M)."""
    vars_ = _d(vars_)
    p, n = vars_.shape
    pairs = _i(pairs).reshape(-1, 2)
    npairs = pairs.shape[0]
    per_pair = np.ndim(alpha) > 0
    alphas = _d(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (npairs,)))
    stats = np.zeros((npairs, 4), dtype=np.float64)
    info = np.zeros((npairs, 6), dtype=np.int32)
    status = np.zeros(npairs, dtype=np.int32)
    M = None
    offs = None
    if want_M:
        fin = np.isfinite(vars_)
        nu = (fin[pairs[:, 0]] & fin[pairs[:, 1]]).sum(axis=1)
        cells = np.array([m_cells(B_of(max(int(m), 1), a)) for m, a in zip(nu, alphas)], dtype=np.int64)
        offs = np.zeros(npairs, dtype=np.int64)
        if npairs:
            offs[1:] = np.cumsum(cells)[:-1]
        M = np.zeros(max(int(cells.sum()), 1), dtype=np.float64)
    args = (_pd(stats), _pi(info), _pi(status), _pd(M) if M is not None else None,
            offs.ctypes.data_as(_lp) if offs is not None else None, int(nthreads))
    if per_pair:
        rc = lib().oracle_score_batch_alphas(_pd(vars_), p, n, _pi(pairs), npairs, _pd(alphas),
                                             float(c), *args)
    else:
        rc = lib().oracle_score_batch(_pd(vars_), p, n, _pi(pairs), npairs, float(alpha),
                                      float(c), *args)
    if rc != 0:
        raise ValueError("oracle_score_batch: " + STATUS.get(rc, str(rc)))
    out = {"stats": stats, "info": info, "status": status}
    if want_M:
        out["M"] = M
        out["M_offsets"] = offs
    return out


def pearson(x, y):
    """Pearson rho over the samples where x and y are both finite (Fig. 1;
    reading R11): returns (rho, n_used); rho is NaN when fewer than two
    samples remain or a variance is zero."""
    x, y = _d(x), _d(y)
    assert len(x) == len(y)
    m = np.zeros(1, dtype=np.int32)
    r = lib().oracle_pearson(_pd(x), _pd(y), len(x), _pi(m))
    return float(r), int(m[0])


def nonlinearity(mic, rho):
    """The non-linearity index MIC - rho^2 (reading R11)."""
    return float(mic) - float(rho) * float(rho)


def max_threads():
    return lib().oracle_max_threads()
