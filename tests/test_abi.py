"""The C ABI library loads and exports every entry point that include/gmine.h
declares; host-only calls behave as documented (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1208_4271_gb300 import build as libbuild
from paper_1208_4271_gb300 import gmine

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gmine.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gmine_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return gmine.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_abi_version_and_struct_sizes(lib):
    assert lib.gmine_abi_version() == 3
    assert gmine.SCORE_DTYPE.itemsize == 72
    assert ctypes.sizeof(gmine.Trace) == 120
    assert ctypes.sizeof(gmine.DPChoice) == 24


def test_header_constants_match_the_binding():
    """The status codes and the stage indexes of include/gmine.h are the
    ones the Python binding uses."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "gmine.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (GMINE_\w+) (\d+)", hdr)}
    for name in ("OK", "E_PARAM", "E_TOO_FEW", "E_CONSTANT", "E_NOMEM", "E_ARG", "E_WORKSPACE", "E_CUDA",
                 "E_LIMIT", "E_NODEVICE", "E_TIMEOUT"):
        assert defs["GMINE_" + name] == getattr(gmine, name), name
    assert defs["GMINE_N_STAGES"] == gmine.N_STAGES == len(gmine.STAGE_NAMES)
    for i, stage in enumerate(gmine.STAGE_NAMES):
        assert defs["GMINE_STAGE_" + stage.upper()] == i, stage
    assert defs["GMINE_ABI_VERSION"] == 3


def test_check_param_matches_documented_ranges(lib):
    assert gmine.check_param(0.6, 15.0) == gmine.OK
    assert gmine.check_param(1.0, 0.5) == gmine.OK
    for a, c in [(0.0, 15), (-0.1, 15), (1.01, 15), (0.6, 0.0), (0.6, -1), (0.6, float("inf")),
                 (float("nan"), 15), (0.6, float("nan"))]:
        assert gmine.check_param(a, c) == gmine.E_PARAM
    assert lib.gmine_check_param(None) == gmine.E_ARG


def test_B_and_cells_agree_with_oracle(lib):
    for n in (4, 10, 16, 300, 1000, 1001, 1340, 16384, 100000):
        for a in (0.5, 0.55, 0.6, 0.75, 1.0):
            assert gmine.B_of(n, a) == oracle.B_of(n, a)
    for B in range(0, 200):
        assert gmine.m_cells(B) == oracle.m_cells(B)


def test_strerror_texts(lib):
    for s in range(0, 11):
        assert isinstance(gmine.strerror(s), str) and gmine.strerror(s)
    assert "unknown" in gmine.strerror(12345)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(gmine, "_lib", None)
    monkeypatch.setattr(gmine, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        gmine.lib()


def test_pearson_batch_argument_checks(lib):
    vp = ctypes.c_void_p
    dummy = vp(16)  # never dereferenced: every call below fails its checks first
    assert lib.gmine_pearson_batch(None, 2, 10, dummy, 1, None, dummy, None, None) == gmine.E_ARG
    assert lib.gmine_pearson_batch(dummy, 2, 10, None, 1, None, dummy, None, None) == gmine.E_ARG
    assert lib.gmine_pearson_batch(dummy, 2, 10, dummy, 1, None, None, None, None) == gmine.E_ARG
    # the non-linearity index needs the scores of the same pairs
    assert lib.gmine_pearson_batch(dummy, 2, 10, dummy, 1, None, dummy, dummy, None) == gmine.E_ARG
    assert lib.gmine_pearson_batch(dummy, -1, 10, dummy, 1, None, dummy, None, None) == gmine.E_ARG
    # nothing to do is success without touching a device
    assert lib.gmine_pearson_batch(None, 0, 0, None, 0, None, None, None, None) == gmine.OK


def test_uneven_batch_argument_checks(lib):
    vp = ctypes.c_void_p
    dummy = vp(16)  # never dereferenced: every call below fails its checks first
    cells, ws = ctypes.c_int64(0), ctypes.c_int64(0)
    good = np.array([0.6, 0.75])
    bad = np.array([0.6, 1.5])
    many = np.linspace(0.3, 0.9, 9)
    plan = lib.gmine_plan_uneven
    assert plan(2, 100, 1, bad.ctypes.data_as(vp), 2, 15.0, 0, ctypes.byref(cells), ctypes.byref(ws)) == gmine.E_PARAM
    assert plan(2, 100, 1, good.ctypes.data_as(vp), 2, -1.0, 0, ctypes.byref(cells), ctypes.byref(ws)) == gmine.E_PARAM
    assert plan(2, 100, 1, many.ctypes.data_as(vp), 9, 15.0, 0, ctypes.byref(cells), ctypes.byref(ws)) == gmine.E_LIMIT
    assert plan(2, 100, 1, None, 1, 15.0, 0, ctypes.byref(cells), ctypes.byref(ws)) == gmine.E_ARG
    assert plan(2, 100, 1, good.ctypes.data_as(vp), 0, 15.0, 0, ctypes.byref(cells), ctypes.byref(ws)) == gmine.E_ARG
    run = lib.gmine_compute_batch_uneven
    # NULL inputs, a missing alpha index array with several alphas, per-task trace arrays
    assert run(None, 2, 10, dummy, 1, good.ctypes.data_as(vp), 2, dummy, 15.0, 0, dummy, 1 << 20,
               dummy, None, None, None) == gmine.E_ARG
    assert run(dummy, 2, 10, dummy, 1, good.ctypes.data_as(vp), 2, None, 15.0, 0, dummy, 1 << 20,
               dummy, None, None, None) == gmine.E_ARG
    tr = gmine.Trace(dummy, None, None, None, 0, 0, None, None, 0, 0, None, None, None, None, None, 0, 0)
    assert run(dummy, 2, 10, dummy, 1, good.ctypes.data_as(vp), 2, dummy, 15.0, 0, dummy, 1 << 20,
               dummy, None, ctypes.byref(tr), None) == gmine.E_ARG


def test_oracle_per_pair_alpha_batch_equals_single():
    rng = np.random.default_rng(4)
    V = rng.normal(size=(8, 150))
    V[3, ::5] = np.nan
    P = np.array([[0, 1], [2, 3], [4, 5], [6, 7]], dtype=np.int32)
    alphas = np.array([0.55, 0.6, 0.75, 0.6])
    out = oracle.score_batch(V, P, alphas, 15.0, nthreads=2, want_M=True)
    for i, (a, b) in enumerate(P):
        r = oracle.score_pair(V[a], V[b], alphas[i], 15.0)
        assert out["stats"][i].tolist() == [r["mic"], r["mas"], r["mev"], r["mcn"]]
        assert out["info"][i, 1] == oracle.B_of(r["n_used"], alphas[i])
        off = out["M_offsets"][i]
        assert np.array_equal(out["M"][off:off + r["m_cells"]], r["M"])
