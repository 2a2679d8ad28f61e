"""Python binding of libgmine (include/gmine.h): argument marshalling only.

Every computation runs in the CUDA library; this module passes pointers and
sizes.  PyTorch provides device memory and streams.  There is no fallback:
if libgmine.so is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmine.so")

(OK, E_PARAM, E_TOO_FEW, E_CONSTANT, E_NOMEM, E_ARG, E_WORKSPACE, E_CUDA, E_LIMIT, E_NODEVICE,
 E_TIMEOUT) = range(11)
PLAIN_FP64 = 0
FP32_DP_FP64_RESCORE = 1
PLAN_HOST_STAGING = 1
PLAN_TRACE = 2

SCORE_DTYPE = np.dtype([("mic", "<f8"), ("mas", "<f8"), ("mev", "<f8"), ("mcn", "<f8"),
                        ("m_offset", "<i8"), ("n_used", "<i4"), ("B", "<i4"),
                        ("m_cells", "<i4"), ("mcn_xy", "<i4"), ("status", "<i4"),
                        ("yhat_x", "<i4"), ("yhat_y", "<i4"), ("reserved", "<i4")])
assert SCORE_DTYPE.itemsize == 72


class GmineError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, strerror(status), status))


class Param(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("c", ctypes.c_double)]


class Trace(ctypes.Structure):
    _fields_ = [("d_k", ctypes.c_void_p), ("d_yhat", ctypes.c_void_p),
                ("d_clumps", ctypes.c_void_p), ("d_sc_ends", ctypes.c_void_p),
                ("sc_stride", ctypes.c_int32), ("cut_stride", ctypes.c_int32),
                ("d_cuts", ctypes.c_void_p), ("d_I", ctypes.c_void_p),
                ("I_stride", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("d_counters", ctypes.c_void_p), ("h_dp_ms", ctypes.c_void_p),
                ("h_dp_launches", ctypes.c_void_p), ("h_kernel_launches", ctypes.c_void_p),
                ("h_launch_ms", ctypes.c_void_p), ("launch_cap", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("h_stage_ms", ctypes.c_void_p)]


N_STAGES = 6
STAGE_NAMES = ("setup", "pairs", "equi", "partition", "dp", "final")


DP_BLOCKED, DP_WARP, DP_MID, DP_SMALL, DP_TWO = range(5)
DP_KIND_NAMES = {DP_BLOCKED: "blocked", DP_WARP: "warp", DP_MID: "mid", DP_SMALL: "small", DP_TWO: "two"}


class DPChoice(ctypes.Structure):
    _fields_ = [("ylo", ctypes.c_int32), ("yhi", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("smem", ctypes.c_int32), ("lev", ctypes.c_int32)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def lib():
    """The loaded libgmine; raises if it is missing (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgmine.so not built: run __graft_entry__.build() "
                               "(paper_1208_4271_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        L.gmine_abi_version.restype = ctypes.c_int
        L.gmine_check_param.argtypes = [ctypes.POINTER(Param)]
        L.gmine_strerror.argtypes = [ctypes.c_int]
        L.gmine_strerror.restype = ctypes.c_char_p
        L.gmine_B.argtypes = [_i64, ctypes.c_double]
        L.gmine_m_cells.argtypes = [_i32]
        L.gmine_m_cells.restype = _i64
        L.gmine_plan.argtypes = [_i64, _i64, _i64, ctypes.POINTER(Param), _i32, _i32,
                                 ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
        L.gmine_compute_batch.argtypes = [_vp, _i64, _i64, _vp, _i64, ctypes.POINTER(Param), _i32,
                                          _vp, _i64, _vp, _vp, _vp]
        L.gmine_compute_batch_ex.argtypes = [_vp, _i64, _i64, _vp, _i64, ctypes.POINTER(Param),
                                             _i32, _vp, _i64, _vp, _vp, ctypes.POINTER(Trace), _vp]
        L.gmine_compute_batch_host.argtypes = [_vp, _i64, _i64, _vp, _i64, ctypes.POINTER(Param),
                                               _i32, _vp, _i64, _vp, _vp, _vp]
        L.gmine_compute_batch_static.argtypes = [_vp, _i64, _i64, _vp, _i64, ctypes.POINTER(Param),
                                                 _i32, _vp, _vp, _vp]
        L.gmine_plan_uneven.argtypes = [_i64, _i64, _i64, _vp, _i32, ctypes.c_double, _i32,
                                        ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
        L.gmine_compute_batch_uneven.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i32, _vp,
                                                 ctypes.c_double, _i32, _vp, _i64, _vp, _vp,
                                                 ctypes.POINTER(Trace), _vp]
        L.gmine_dp_groups.argtypes = [_i64, ctypes.c_double, ctypes.c_double, _i32,
                                      ctypes.POINTER(DPChoice), _i32, ctypes.POINTER(_i32)]
        L.gmine_set_dp_choices.argtypes = [_i64, ctypes.c_double, ctypes.c_double, _i32,
                                           ctypes.POINTER(DPChoice), _i32]
        L.gmine_rank.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp]
        L.gmine_equipartition.argtypes = [_vp, _i64, _i64, _i32, _vp, _vp, _vp, _i64, _vp]
        L.gmine_score_pair_host.argtypes = [_vp, _vp, _i64, ctypes.POINTER(Param), _i32, _vp, _vp]
        L.gmine_pearson_batch.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _vp]
        for f in ("gmine_mic", "gmine_mas", "gmine_mev", "gmine_mcn"):
            getattr(L, f).argtypes = [_vp]
            getattr(L, f).restype = ctypes.c_double
        _lib = L
    return _lib


def strerror(status):
    try:
        return lib().gmine_strerror(int(status)).decode()
    except Exception:  # the library itself is missing
        return "status %d" % status


def _check(rc, where):
    if rc != OK:
        raise GmineError(rc, where)


def B_of(n, alpha):
    return int(lib().gmine_B(int(n), float(alpha)))


def m_cells(B):
    return int(lib().gmine_m_cells(int(B)))


def check_param(alpha, c):
    return lib().gmine_check_param(ctypes.byref(Param(alpha, c)))


def plan(p, n, n_pairs, alpha=0.6, c=15.0, precision=PLAIN_FP64, flags=0):
    cells = _i64(0)
    ws = _i64(0)
    _check(lib().gmine_plan(int(p), int(n), int(n_pairs), ctypes.byref(Param(alpha, c)),
                            int(precision), int(flags), ctypes.byref(cells), ctypes.byref(ws)),
           "gmine_plan")
    return int(cells.value), int(ws.value)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Workspace:
    """A device workspace sized by gmine_plan, reusable across calls of the
    same shape."""

    def __init__(self, p, n, n_pairs, alpha=0.6, c=15.0, precision=PLAIN_FP64, flags=0,
                 device="cuda"):
        import torch
        self.cells, self.nbytes = plan(p, n, n_pairs, alpha, c, precision, flags)
        self.buf = torch.empty(max(self.nbytes, 1), dtype=torch.uint8, device=device)

    @property
    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())


def trace_strides(n, alpha, c):
    """Strides of the per-task trace buffers for a batch of n samples."""
    B = B_of(n, alpha)
    xmax = B // 2
    kmax = 1
    for y in range(2, B // 2 + 1):
        x = B // y
        kh = max(int(np.floor(c * x)), 1)
        kmax = max(kmax, min(kh, n))
    return {"B": B, "R": max(B // 2 - 1, 0), "sc_stride": kmax + 1,
            "cut_stride": max(xmax * (xmax - 1) // 2, 1), "I_stride": max(xmax - 1, 1)}


def alloc_trace(n_pairs, n, alpha, c, device="cuda"):
    """Device buffers for gmine_trace; returns (Trace struct, dict of tensors)."""
    import torch
    st = trace_strides(n, alpha, c)
    tasks = max(2 * st["R"] * n_pairs, 1)
    t = {"k": torch.full((tasks,), -7, dtype=torch.int32, device=device),
         "yhat": torch.full((tasks,), -7, dtype=torch.int32, device=device),
         "clumps": torch.full((tasks,), -7, dtype=torch.int32, device=device),
         "sc_ends": torch.full((tasks, st["sc_stride"]), -7, dtype=torch.int32, device=device),
         "cuts": torch.full((tasks, st["cut_stride"]), -7, dtype=torch.int32, device=device),
         "I": torch.full((tasks, st["I_stride"]), float("nan"), dtype=torch.float64, device=device)}
    t["counters"] = torch.zeros(2, dtype=torch.int64, device=device)
    tr = Trace(_dptr(t["k"]), _dptr(t["yhat"]), _dptr(t["clumps"]), _dptr(t["sc_ends"]),
               st["sc_stride"], st["cut_stride"], _dptr(t["cuts"]), _dptr(t["I"]),
               st["I_stride"], 0, _dptr(t["counters"]), None, None, None, None, 0, 0)
    t.update(st)
    return tr, t


class Measure:
    """Counters and DP kernel timing of one batch call (gmine_trace without
    the per-task tables): subtract-and-max steps, tasks, summed DP kernel
    milliseconds measured with CUDA events on the call's stream, and the
    milliseconds of each DP launch (up to launch_cap) and of each stage of
    the call (stage_ms)."""

    def __init__(self, device="cuda", launch_cap=4096):
        import torch
        self.counters = torch.zeros(2, dtype=torch.int64, device=device)
        self._ms = ctypes.c_double(0.0)
        self._launches = ctypes.c_int32(0)
        self._kernels = ctypes.c_int32(0)
        self._launch_ms = np.zeros(launch_cap, dtype=np.float32)
        self._stage_ms = np.zeros(N_STAGES, dtype=np.float64)
        self.trace = Trace(None, None, None, None, 0, 0, None, None, 0, 0,
                           _dptr(self.counters), ctypes.cast(ctypes.byref(self._ms), ctypes.c_void_p),
                           ctypes.cast(ctypes.byref(self._launches), ctypes.c_void_p),
                           ctypes.cast(ctypes.byref(self._kernels), ctypes.c_void_p),
                           self._launch_ms.ctypes.data_as(ctypes.c_void_p), launch_cap, 0,
                           self._stage_ms.ctypes.data_as(ctypes.c_void_p))

    @property
    def stage_ms(self):
        """Milliseconds of each stage of the last call (STAGE_NAMES order)."""
        return dict(zip(STAGE_NAMES, (float(v) for v in self._stage_ms)))

    @property
    def launch_ms(self):
        return self._launch_ms[:min(self._launches.value, self._launch_ms.size)].copy()

    @property
    def dp_ms(self):
        return self._ms.value

    @property
    def dp_launches(self):
        return self._launches.value

    @property
    def kernel_launches(self):
        return self._kernels.value


def dp_groups(n, alpha=0.6, c=15.0, precision=PLAIN_FP64):
    """The DP launch groups planned on the current device: a list of dicts
    (ylo, yhi, kind, threads, smem, lev)."""
    cap = 64
    arr = (DPChoice * cap)()
    cnt = _i32(0)
    _check(lib().gmine_dp_groups(int(n), float(alpha), float(c), int(precision), arr, cap,
                                 ctypes.byref(cnt)), "gmine_dp_groups")
    return [{f: int(getattr(arr[i], f)) for f, _ in DPChoice._fields_} for i in range(min(cnt.value, cap))]


def set_dp_choices(n, alpha, c, precision, choices):
    """Tuned (ylo, yhi, kind, threads) choices for batches of this shape
    (an empty list removes them)."""
    arr = (DPChoice * max(len(choices), 1))()
    for i, ch in enumerate(choices):
        arr[i] = DPChoice(int(ch["ylo"]), int(ch["yhi"]), int(ch["kind"]), int(ch["threads"]), 0, 0)
    _check(lib().gmine_set_dp_choices(int(n), float(alpha), float(c), int(precision), arr, len(choices)),
           "gmine_set_dp_choices")


def compute_batch(vars_, pairs, alpha=0.6, c=15.0, precision=PLAIN_FP64, want_M=True,
                  workspace=None, trace=None, stream=None):
    """All pairs on the device.  vars_: CUDA float64 [p, n]; pairs: CUDA int32
    [n_pairs, 2].  Returns (scores as a CUDA uint8 [n_pairs, 72] tensor, M or
    None).  Asynchronous on the stream; see scores_to_numpy."""
    import torch
    assert vars_.is_cuda and vars_.dtype == torch.float64 and vars_.is_contiguous()
    assert pairs.is_cuda and pairs.dtype == torch.int32 and pairs.is_contiguous()
    p, n = vars_.shape
    n_pairs = pairs.shape[0]
    flags = PLAN_TRACE if trace is not None else 0
    if workspace is None:
        workspace = Workspace(p, n, n_pairs, alpha, c, precision, flags, device=vars_.device)
    scores = torch.empty((max(n_pairs, 1), SCORE_DTYPE.itemsize), dtype=torch.uint8, device=vars_.device)
    M = None
    if want_M:
        M = torch.zeros(max(n_pairs * workspace.cells, 1), dtype=torch.float64, device=vars_.device)
    prm = Param(alpha, c)
    if trace is None:
        rc = lib().gmine_compute_batch(_dptr(vars_), p, n, _dptr(pairs), n_pairs, ctypes.byref(prm),
                                       int(precision), workspace.ptr, workspace.nbytes,
                                       _dptr(scores), _dptr(M), _stream_ptr(stream))
    else:
        rc = lib().gmine_compute_batch_ex(_dptr(vars_), p, n, _dptr(pairs), n_pairs,
                                          ctypes.byref(prm), int(precision), workspace.ptr,
                                          workspace.nbytes, _dptr(scores), _dptr(M),
                                          ctypes.byref(trace), _stream_ptr(stream))
    _check(rc, "gmine_compute_batch")
    return scores[:n_pairs], M


def alpha_table(alphas):
    """Per-pair alpha values -> (distinct values as a float64 array, uint8
    index of each pair into it)."""
    a = np.asarray(alphas, dtype=np.float64).reshape(-1)
    vals, idx = np.unique(a, return_inverse=True)
    return np.ascontiguousarray(vals), idx.astype(np.uint8)


def plan_uneven(p, n, n_pairs, alpha_values, c=15.0, precision=PLAIN_FP64):
    vals = np.ascontiguousarray(alpha_values, dtype=np.float64).reshape(-1)
    cells = _i64(0)
    ws = _i64(0)
    _check(lib().gmine_plan_uneven(int(p), int(n), int(n_pairs), vals.ctypes.data_as(_vp), len(vals),
                                   float(c), int(precision), ctypes.byref(cells), ctypes.byref(ws)),
           "gmine_plan_uneven")
    return int(cells.value), int(ws.value)


class UnevenWorkspace:
    """A device workspace for gmine_compute_batch_uneven."""

    def __init__(self, p, n, n_pairs, alpha_values, c=15.0, precision=PLAIN_FP64, device="cuda"):
        import torch
        self.cells, self.nbytes = plan_uneven(p, n, n_pairs, alpha_values, c, precision)
        self.buf = torch.empty(max(self.nbytes, 1), dtype=torch.uint8, device=device)

    @property
    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())


def compute_batch_uneven(vars_, pairs, alphas, c=15.0, precision=PLAIN_FP64, want_M=True,
                         workspace=None, measure=None, stream=None):
    """Pairs of uneven size, each with its own alpha (gmine_compute_batch_uneven).
    vars_: CUDA float64 [p, n] (NaN-padded); pairs: CUDA int32 [n_pairs, 2];
    alphas: one alpha per pair (host sequence).  Returns (scores, M)."""
    import torch
    assert vars_.is_cuda and vars_.dtype == torch.float64 and vars_.is_contiguous()
    assert pairs.is_cuda and pairs.dtype == torch.int32 and pairs.is_contiguous()
    p, n = vars_.shape
    n_pairs = pairs.shape[0]
    vals, idx = alpha_table(alphas)
    assert idx.size == n_pairs
    if workspace is None:
        workspace = UnevenWorkspace(p, n, n_pairs, vals, c, precision, device=vars_.device)
    aidx = torch.from_numpy(idx).to(vars_.device)
    scores = torch.empty((max(n_pairs, 1), SCORE_DTYPE.itemsize), dtype=torch.uint8, device=vars_.device)
    M = None
    if want_M:
        M = torch.zeros(max(n_pairs * workspace.cells, 1), dtype=torch.float64, device=vars_.device)
    rc = lib().gmine_compute_batch_uneven(_dptr(vars_), p, n, _dptr(pairs), n_pairs,
                                          vals.ctypes.data_as(_vp), len(vals), _dptr(aidx), float(c),
                                          int(precision), workspace.ptr, workspace.nbytes,
                                          _dptr(scores), _dptr(M),
                                          ctypes.byref(measure.trace) if measure is not None else None,
                                          _stream_ptr(stream))
    _check(rc, "gmine_compute_batch_uneven")
    return scores[:n_pairs], M


def compute_batch_static(vars_, pairs, alpha=0.6, c=15.0, precision=PLAIN_FP64, want_M=True,
                         stream=None):
    """gmine_compute_batch_static: the batch with the library's own fixed
    scratch array (no workspace allocated anywhere).  Returns (status, scores,
    M); status GMINE_E_WORKSPACE means the batch needs more than the array."""
    import torch
    assert vars_.is_cuda and vars_.dtype == torch.float64 and vars_.is_contiguous()
    assert pairs.is_cuda and pairs.dtype == torch.int32 and pairs.is_contiguous()
    p, n = vars_.shape
    n_pairs = pairs.shape[0]
    cells = m_cells(B_of(max(n, 1), alpha)) if n > 0 else 1
    scores = torch.zeros((max(n_pairs, 1), SCORE_DTYPE.itemsize), dtype=torch.uint8,
                         device=vars_.device)
    M = torch.zeros(max(n_pairs * max(cells, 1), 1), dtype=torch.float64,
                    device=vars_.device) if want_M else None
    rc = lib().gmine_compute_batch_static(_dptr(vars_), p, n, _dptr(pairs), n_pairs,
                                          ctypes.byref(Param(alpha, c)), int(precision),
                                          _dptr(scores), _dptr(M), _stream_ptr(stream))
    return rc, scores[:n_pairs], M


def pearson_batch(vars_, pairs, scores=None, stream=None):
    """gmine_pearson_batch: Pearson rho of each pair over its finite samples
    and, when `scores` (from compute_batch on the same pairs) is given, the
    non-linearity index MIC - rho^2.  Returns (rho, nonlin or None), CUDA
    float64 [n_pairs] tensors; asynchronous on the stream."""
    import torch
    assert vars_.is_cuda and vars_.dtype == torch.float64 and vars_.is_contiguous()
    assert pairs.is_cuda and pairs.dtype == torch.int32 and pairs.is_contiguous()
    p, n = vars_.shape
    n_pairs = pairs.shape[0]
    rho = torch.empty(max(n_pairs, 1), dtype=torch.float64, device=vars_.device)
    nonlin = None
    if scores is not None:
        assert scores.is_cuda and scores.shape[0] == n_pairs and scores.is_contiguous()
        nonlin = torch.empty(max(n_pairs, 1), dtype=torch.float64, device=vars_.device)
    _check(lib().gmine_pearson_batch(_dptr(vars_), p, n, _dptr(pairs), n_pairs, _dptr(scores),
                                     _dptr(rho), _dptr(nonlin), _stream_ptr(stream)),
           "gmine_pearson_batch")
    return rho[:n_pairs], (nonlin[:n_pairs] if nonlin is not None else None)


def scores_to_numpy(scores):
    """uint8 [n_pairs, 72] (device or host tensor) -> structured numpy array."""
    a = scores.cpu().numpy() if hasattr(scores, "cpu") else np.asarray(scores)
    return np.ascontiguousarray(a).view(SCORE_DTYPE).reshape(-1)


def compute_batch_host(vars_np, pairs_np, alpha=0.6, c=15.0, precision=PLAIN_FP64, want_M=True,
                       workspace=None, stream=None, out_scores=None, out_M=None):
    """Host arrays in and out (gmine_compute_batch_host): copies inside."""
    vars_np = np.ascontiguousarray(vars_np, dtype=np.float64)
    pairs_np = np.ascontiguousarray(pairs_np, dtype=np.int32).reshape(-1, 2)
    p, n = vars_np.shape
    n_pairs = pairs_np.shape[0]
    if workspace is None:
        workspace = Workspace(p, n, n_pairs, alpha, c, precision, PLAN_HOST_STAGING)
    scores = out_scores if out_scores is not None else np.zeros(max(n_pairs, 1), dtype=SCORE_DTYPE)
    M = None
    if want_M:
        M = out_M if out_M is not None else np.zeros(max(n_pairs * workspace.cells, 1))
    prm = Param(alpha, c)
    rc = lib().gmine_compute_batch_host(vars_np.ctypes.data_as(_vp), p, n,
                                        pairs_np.ctypes.data_as(_vp), n_pairs, ctypes.byref(prm),
                                        int(precision), workspace.ptr, workspace.nbytes,
                                        scores.ctypes.data_as(_vp),
                                        M.ctypes.data_as(_vp) if M is not None else None,
                                        _stream_ptr(stream))
    _check(rc, "gmine_compute_batch_host")
    return scores[:n_pairs], M


def rank(vars_, stream=None):
    """Tie-aware sort of every variable: (perm, dense rank, groups)."""
    import torch
    p, n = vars_.shape
    ws = Workspace(p, n, 0)
    perm = torch.empty((p, n), dtype=torch.int32, device=vars_.device)
    rk = torch.empty((p, n), dtype=torch.int32, device=vars_.device)
    groups = torch.empty((max(p, 1),), dtype=torch.int32, device=vars_.device)
    _check(lib().gmine_rank(_dptr(vars_), p, n, _dptr(perm), _dptr(rk), _dptr(groups), ws.ptr,
                            ws.nbytes, _stream_ptr(stream)), "gmine_rank")
    return perm, rk, groups[:p]


def equipartition(vars_, y, stream=None):
    """EquipartitionYAxis of every variable into y rows: (Q, yhat)."""
    import torch
    p, n = vars_.shape
    ws = Workspace(p, n, 0)
    Q = torch.empty((p, n), dtype=torch.int32, device=vars_.device)
    yh = torch.empty((max(p, 1),), dtype=torch.int32, device=vars_.device)
    _check(lib().gmine_equipartition(_dptr(vars_), p, n, int(y), _dptr(Q), _dptr(yh), ws.ptr,
                                     ws.nbytes, _stream_ptr(stream)), "gmine_equipartition")
    return Q, yh[:p]


def score_pair(x, y, alpha=0.6, c=15.0, precision=PLAIN_FP64):
    """mine_compute_score for one pair of host vectors (synchronous)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(x)
    B = B_of(max(n, 1), alpha)
    out = np.zeros(1, dtype=SCORE_DTYPE)
    M = np.zeros(max(m_cells(B), 1))
    _check(lib().gmine_score_pair_host(x.ctypes.data_as(_vp), y.ctypes.data_as(_vp), n,
                                       ctypes.byref(Param(alpha, c)), int(precision),
                                       out.ctypes.data_as(_vp), M.ctypes.data_as(_vp)),
           "gmine_score_pair_host")
    s = out[0]
    return {"status": int(s["status"]), "mic": float(s["mic"]), "mas": float(s["mas"]),
            "mev": float(s["mev"]), "mcn": float(s["mcn"]), "mcn_xy": int(s["mcn_xy"]),
            "n_used": int(s["n_used"]), "B": int(s["B"]), "m_cells": int(s["m_cells"]),
            "M": M[:int(s["m_cells"])].copy()}
