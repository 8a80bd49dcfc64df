"""The C-ABI library loads and exports every function include/bbx.h declares;
argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_1605_06015_gb300 import bbx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bbx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bbx_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(bbx.lib(), n), n


def test_status_strings():
    for code in range(-9, 1):
        assert bbx.bbx_status_string(code) not in ("", "unknown status")
    assert bbx.bbx_status_string(-100) == "unknown status"


def test_argument_errors_without_gpu():
    L = bbx.lib()
    g = ctypes.c_void_p()
    assert L.bbx_create_grid(None, 4, 4, 4, 1.0, None, None) == bbx.BBX_ERR_ARG
    assert L.bbx_create_grid(ctypes.byref(g), 0, 4, 4, 1.0, None, None) == bbx.BBX_ERR_ARG
    assert L.bbx_create_grid(ctypes.byref(g), 4, 4, 4, -1.0, None, None) == bbx.BBX_ERR_ARG
    assert L.bbx_create_grid(ctypes.byref(g), 2048, 2048, 1024, 1.0, None, None) == bbx.BBX_ERR_ARG
    assert L.bbx_step(None, 0.1, 1) == bbx.BBX_ERR_ARG
    assert L.bbx_read_state(None, 0, None, 0) == bbx.BBX_ERR_ARG
    assert L.bbx_set_fibres(None, None, 1.0, 1.0) == bbx.BBX_ERR_ARG
    assert L.bbx_set_wsum_elision(None, 1) == bbx.BBX_ERR_ARG
    L.bbx_destroy_grid(None)


def test_noalloc_total_refuses_bad_arguments_without_gpu():
    # every refusal of bbx_total_noalloc returns before any CUDA call; the
    # pointers are dummies that are never dereferenced
    L = bbx.lib()
    f = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x2000)
    T = L.bbx_total_noalloc
    assert T(None, None, 8, 8, 8, 8, out, None) == bbx.BBX_ERR_ARG          # no field
    assert T(f, None, 8, 8, 8, 8, None, None) == bbx.BBX_ERR_ARG            # no output
    assert T(f, None, 8, 8, 8, 7, out, None) == bbx.BBX_ERR_ARG             # pitch < nx
    assert T(f, None, 0, 8, 8, 8, out, None) == bbx.BBX_ERR_ARG             # empty
    assert T(f, None, 8, -1, 8, 8, out, None) == bbx.BBX_ERR_ARG
    assert T(f, None, 1 << 15, 1 << 14, 2, 1 << 15, out, None) == bbx.BBX_ERR_ARG  # 2^29 > 2^28 nodes


def test_binding_names_match_the_c_abi():
    for n in _declared():
        assert callable(getattr(bbx, n)), n
