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
