"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lisa_td.h declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2501_08261_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lisa_\w+|flow_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert "lisa_td_loglike_batch" in names and len(names) >= 8
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(declared_functions()) <= set(api.EXPORTS)


def test_config_struct_layout_matches_header():
    # 5 doubles / int64 then 9 int32 fields, padded to the 8-byte alignment
    assert ctypes.sizeof(api.Config) == 5 * 8 + 9 * 4 + 4
    assert api.Config.tdi_gen.offset == 40 and api.Config.max_walkers.offset == 68
    assert api.Config.tdi_nested.offset == 72


def test_argument_errors_need_no_gpu(libpath):
    lib = api.load_library(libpath)
    h = ctypes.c_void_p()
    bad = api.make_config(dt=5.0, n=17280, tdi_gen=16)
    rc = lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None)
    assert rc == -1 and b"tdi_gen" in lib.lisa_td_last_error()
    bad = api.make_config(dt=5.0, n=17281)
    rc = lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None)
    assert rc == -1 and b"2^a 3^b" in lib.lisa_td_last_error()
    bad = api.make_config(dt=5.0, n=17280, tdi_nested=2)
    rc = lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None)
    assert rc == -1 and b"tdi_nested" in lib.lisa_td_last_error()
    bad = api.make_config(dt=5.0, n=17280, lagrange_order=9)
    assert lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    assert lib.lisa_td_create(None, ctypes.byref(bad), None) == -1
    assert lib.lisa_td_loglike_batch(None, None, 1, None, None, None) == -1
    # heterodyned likelihood: NULL context / arguments are refused before any device work
    assert lib.lisa_td_het_setup(None, None, None, 2, None) == -1
    assert b"NULL" in lib.lisa_td_last_error()
    assert lib.lisa_td_het_loglike(None, None, 1, None, None, None) == -1
    assert lib.lisa_td_het_deltas(None, None, 1, None, None) == -1
    assert lib.lisa_td_het_aet(None, None, 1, None, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.load_library(str(tmp_path / "nope.so"))


def test_flow_and_sampler_argument_errors_need_no_gpu(libpath):
    lib = api.load_library(libpath)
    h = ctypes.c_void_p()
    idx = (ctypes.c_int32 * 15)(*range(15))
    perm = (ctypes.c_int32 * 15)(*range(15))
    assert lib.flow_create(ctypes.byref(h), 16, 1, 128, 64, idx, perm, None) == -1
    assert lib.flow_create(ctypes.byref(h), 15, 1, 64, 64, idx, perm, None) == -1
    assert b"128" in lib.lisa_td_last_error()
    bad = (ctypes.c_int32 * 15)(*([0] * 15))
    assert lib.flow_create(ctypes.byref(h), 15, 1, 128, 64, bad, perm, None) == -1
    assert lib.lisa_fisher_npoints(15) == 451
    assert lib.lisa_cholesky(None, None, 3, None, None, None) == -1


def test_orbit_table_checks_need_no_gpu(libpath):
    """lisa_td_create_orbits validates the table on the host before any CUDA
    call: NULL, too few rows, a grid not covered, non-physical arms."""
    import numpy as np
    from paper_2501_08261_gb300 import workloads
    lib = api.load_library(libpath)
    cfg = api.make_config(dt=5.0, n=17280, orbit=2, tdi_gen=20)
    h = ctypes.c_void_p()
    assert lib.lisa_td_create_orbits(ctypes.byref(h), ctypes.byref(cfg), None, None) == -1
    good = workloads.orbit_table_positions(-7200.0, 3600.0, 40, 3)

    def call(t0, dt, pos, c=cfg):
        arr = np.ascontiguousarray(pos)
        tab = api.OrbitTable(t0, dt, arr.shape[0], arr.ctypes.data)
        return lib.lisa_td_create_orbits(ctypes.byref(h), ctypes.byref(c), ctypes.byref(tab), None)
    assert call(-7200.0, 3600.0, good[:7]) == -1                      # rows < 8
    assert b"8 rows" in lib.lisa_td_last_error()
    assert call(-60.0, 3600.0, good) == -1                            # starts too late
    assert call(-7200.0, 3600.0, good[:20]) == -1                     # ends before the grid
    assert b"cover" in lib.lisa_td_last_error()
    bad = good.copy()
    bad[5, 1] *= 1.01                                                 # a craft 0.01 AU off
    assert call(-7200.0, 3600.0, bad) == -1
    assert b"arm" in lib.lisa_td_last_error()
    nan = good.copy()
    nan[3, 2, 1] = float("nan")
    assert call(-7200.0, 3600.0, nan) == -1
    kind1 = api.make_config(dt=5.0, n=17280, orbit=1)
    assert call(-7200.0, 3600.0, good, kind1) == -1                   # needs orbit_kind 2
    assert lib.lisa_td_create(ctypes.byref(h), ctypes.byref(cfg), None) == -1


def test_allocation_failure_injection_needs_no_gpu(libpath, monkeypatch):
    """LISA_TD_FAIL_ALLOC=0 fails the first workspace allocation before any
    CUDA call: LISA_TD_ENOMEM and a NULL context."""
    lib = api.load_library(libpath)
    cfg = api.make_config(dt=5.0, n=17280)
    h = ctypes.c_void_p(1)
    monkeypatch.setenv("LISA_TD_FAIL_ALLOC", "0")
    assert lib.lisa_td_create(ctypes.byref(h), ctypes.byref(cfg), None) == -2
    assert h.value is None
    assert b"cudaMalloc" in lib.lisa_td_last_error()


def test_binding_refuses_truncated_or_mistyped_tensors():
    """The C ABI takes bare pointers, so the binding checks every tensor before
    its pointer crosses: truncated data ([3][n - 1] for [3][n]), another
    dtype, host memory and non-contiguous views are refused on the host."""
    torch = pytest.importorskip("torch")
    n = 64
    full = torch.zeros((3, n), dtype=torch.float64)
    with pytest.raises(ValueError, match="shape"):
        api._need(full[:, :-1], torch.float64, (3, n), "data")
    with pytest.raises(ValueError, match="shape"):
        api._need(full[:2], torch.float64, (3, n), "data")
    with pytest.raises(TypeError, match="dtype"):
        api._need(full.float(), torch.float64, (3, n), "data")
    with pytest.raises(ValueError, match="CUDA"):
        api._need(full, torch.float64, (3, n), "data")
