"""The C-ABI library loads and exports every entry point include/rf.h declares
(no GPU work: only calls that validate arguments on the host)."""
import ctypes
import os
import re

import pytest

from paper_2502_01157_gb300 import build as B
from paper_2502_01157_gb300 import rf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rf.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"RF_API\s+[\w\s\*]+?\b(rf_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return rf.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("rf_scene_create", "rf_render_fwd", "rf_render_bwd", "rf_trace_cells"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    raw = ctypes.CDLL(B.LIB)
    missing = [n for n in declared_symbols() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(rf.SIGNATURES)


def test_version_and_argument_errors_without_gpu(L):
    assert L.rf_version() == 1
    h = ctypes.c_void_p()
    assert L.rf_scene_create(None, None, ctypes.byref(h)) == 1  # RF_ERR_INVALID_ARG
    assert b"NULL" in L.rf_last_error()
    d = rf.rf_scene_desc()
    d.n_sites = 0
    assert L.rf_scene_create(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert L.rf_render_fwd(None, None, 0, None, None, None, None, None, None, None) == 1
    assert L.rf_scene_destroy(None) == 0
