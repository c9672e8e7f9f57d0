"""CPU checks of the C ABI: the library loads, exports what include/hdp.h
declares, and rejects invalid parameters before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_1509_08197_gb300 as hdp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hdp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1509_08197_gb300 import build
    build.build()
    return hdp.load()


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert "hdp_create" in names and "hdp_match" in names and "hdp_destroy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    assert set(names) == set(hdp.exported_symbols())


def test_default_params(lib):
    p = hdp._Params()
    lib.hdp_default_params(ctypes.byref(p), 1390, 1110, 255)
    assert (p.levels, p.beta_num, p.beta_den) == (4, 95, 100)
    assert abs(p.delta0 - 0.004) < 1e-12 and abs(p.gamma - 25.5) < 1e-6
    lib.hdp_default_params(ctypes.byref(p), 463, 370, 79)
    assert (p.beta_num, p.beta_den) == (3, 5) and abs(p.delta0 - 0.064) < 1e-12


@pytest.mark.parametrize("field,value", [
    ("max_disp", 0), ("max_disp", 256), ("levels", 0), ("levels", 9), ("width", 1), ("alpha", 0.93),
    ("tau_c", 7.1), ("beta_num", 7), ("delta0", 1.5), ("tree", 5), ("storage", 3), ("prefilter", 2),
])
def test_invalid_params_rejected(lib, field, value):
    p = hdp._Params()
    lib.hdp_default_params(ctypes.byref(p), 64, 48, 15)
    if field == "beta_num":
        p.beta_num, p.beta_den = 7, 5
    else:
        setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.hdp_create(ctypes.byref(p), None, ctypes.byref(h)) == hdp.HDP_ERR_ARG
    assert not h.value


def test_null_arguments(lib):
    assert lib.hdp_create(None, None, None) == hdp.HDP_ERR_ARG
    assert lib.hdp_match(None, None) == hdp.HDP_ERR_ARG
    assert lib.hdp_destroy(None) == hdp.HDP_ERR_ARG
    assert lib.hdp_build_trees(None, None, None, 0) == hdp.HDP_ERR_ARG
