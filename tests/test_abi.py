"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point declared in include/mbir.h (no device calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mbir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b([a-z][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("mbir_", "mbmd_", "psps_"))))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["mbir_project", "mbir_backproject", "mbmd_forward_model", "mbmd_gradient", "psps_precondition",
                 "psps_step", "mbir_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2010_01371_gb300 import _abi, _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    wrapped = {s[0] for s in _abi.SIGNATURES}
    assert set(declared_functions()) == wrapped


def test_built_for_sm103a():
    from paper_2010_01371_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.build())


def test_last_error_without_device():
    """Argument validation happens before any device work, so a bad call
    fails cleanly even on a host without a GPU."""
    from paper_2010_01371_gb300 import _abi
    lib = _abi.load()
    h = ctypes.c_void_p()
    st = lib.mbir_plan_create(None, 1, ctypes.byref(h))
    assert st == -1
    assert b"null" in lib.mbir_last_error()
    g = _abi.MbirGeometry(7, 8, 8, 1, 1.0, 1.0, 1.0, 4, 0.0, 3.14, 8, 1, 1.0, 1.0, 0.0, 0.0)
    assert lib.mbir_plan_create(ctypes.byref(g), 1, ctypes.byref(h)) == -1
    assert b"kind" in lib.mbir_last_error()
    Q = (ctypes.c_double * 1)(-1.0)
    S = (ctypes.c_double * 1)(1.0)
    assert lib.mbmd_spectrum_create(1, 1, 1, Q, S, ctypes.byref(h)) == -1
