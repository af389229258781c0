"""CPU checks of the C-ABI library: it loads, exports every declared entry
point, and its enums agree with the binding and the oracle's status names."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bs3.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_23727_gb300 import bs3
    return bs3.load()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(bs3_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("bs3_create_system", "bs3_set_coupling", "bs3_solve", "bs3_destroy_system",
              "bs3_status_string", "bs3_rhs", "bs3_attempt"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2605_23727_gb300 import bs3
    assert sorted(bs3.EXPORTED) == _declared()


def test_enum_values_match_header():
    from paper_2605_23727_gb300 import bs3
    txt = open(HEADER).read()
    for name, val in re.findall(r"BS3_([A-Z0-9_]+)\s*=\s*(\d+)", txt):
        if hasattr(bs3, name):
            assert getattr(bs3, name) == int(val), name


def test_status_strings_and_limits_without_gpu(lib):
    from oracle import bs3 as obs3
    from paper_2605_23727_gb300 import bs3
    for code, name in obs3.STATUS_NAMES.items():
        assert bs3.bs3_status_string(code) == "BS3_" + name
    lim = bs3.bs3_default_limits()
    assert (lim.max_attempts, lim.max_rejects, lim.hmin_factor) == (100000, 85000, 100.0)
    assert lim.wall_limit_s == 5400.0 and lim.slow_limit_s == 2700.0 and lim.slow_fraction == 0.1


def test_create_system_rejects_bad_arguments(lib):
    import ctypes
    from paper_2605_23727_gb300 import bs3
    out = ctypes.c_void_p()
    assert lib.bs3_create_system(7, 10, None, 0, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    assert lib.bs3_create_system(bs3.KURAMOTO, 10, None, 3, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    assert lib.bs3_create_system(bs3.KURAMOTO, 0, None, 0, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    assert lib.bs3_solve(None, 0.0, 1.0, None, 1e-6, 1e-6, 0, 0, None, 0, None, None, 0, None, None) \
        == bs3.ERR_INVALID_ARG
