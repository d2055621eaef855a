"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lisa_td.h declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2501_08261_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lisa_td.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lisa_td_\w+|flow_\w+)\s*\(", src)))


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
    # 5 doubles / int64 then 8 int32 fields, no padding
    assert ctypes.sizeof(api.Config) == 5 * 8 + 8 * 4
    assert api.Config.tdi_gen.offset == 40 and api.Config.max_walkers.offset == 68


def test_argument_errors_need_no_gpu(libpath):
    lib = api.load_library(libpath)
    h = ctypes.c_void_p()
    bad = api.make_config(dt=5.0, n=17280, tdi_gen=16)
    rc = lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None)
    assert rc == -1 and b"tdi_gen" in lib.lisa_td_last_error()
    bad = api.make_config(dt=5.0, n=17281)
    rc = lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None)
    assert rc == -1 and b"2^a 3^b" in lib.lisa_td_last_error()
    bad = api.make_config(dt=5.0, n=17280, lagrange_order=9)
    assert lib.lisa_td_create(ctypes.byref(h), ctypes.byref(bad), None) == -1
    assert lib.lisa_td_create(None, ctypes.byref(bad), None) == -1
    assert lib.lisa_td_loglike_batch(None, None, 1, None, None, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.load_library(str(tmp_path / "nope.so"))
