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


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (compiled with the host C compiler, no GPU)."""
    structs = {n: getattr(rf, n) for n in ("rf_camera", "rf_scene_desc", "rf_render_opts",
                                           "rf_serve_config", "rf_serve_metrics", "rf_fwd_outputs",
                                           "rf_bwd_inputs", "rf_grads")}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for n, cls in structs.items():
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in cls._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    r = subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        n, f, v = ln.split()
        got[(n, f)] = int(v)
    for n, cls in structs.items():
        assert got[(n, "size")] == ctypes.sizeof(cls), n
        for f in cls._fields_:
            assert got[(n, f[0])] == getattr(cls, f[0]).offset, (n, f[0])


def test_walk_record_bytes_without_gpu(L):
    """Host-side sizing of the walk record: 4 warps of 32 rays per 16x8 tile,
    24 bytes per step (exit id, t1, density, three colour values), launches
    of up to 16 cameras concatenated."""
    from paper_2502_01157_gb300 import scenes as S
    cams = [S.pinhole(w, h, 60.0) for w, h in [(1920, 1080), (17, 9), (1, 1)] * 7]   # 21 cameras
    tiles = sum(((c.width + 15) // 16) * ((c.height + 7) // 8) for c in cams)
    for steps in (1, 7, 384):
        assert rf.walk_record_bytes(cams, steps) == tiles * 4 * steps * 32 * 24
    ca = rf.camera_array(cams)
    assert L.rf_walk_record_bytes(ca, len(ca), 0) == 0
    assert L.rf_walk_record_bytes(None, 3, 8) == 0


def test_null_handles_and_pointers_are_rejected_on_the_host(L):
    """Every entry point that takes a handle or a required pointer returns
    RF_ERR_INVALID_ARG for NULL before it touches the device, and the
    destroy calls accept NULL."""
    from paper_2502_01157_gb300 import scenes as S
    INVALID = 1
    cam = rf.camera_array([S.pinhole(8, 8, 60.0)])
    opts = rf.opts_struct()
    n64, e64 = ctypes.c_int64(), ctypes.c_int64()
    calls = {
        "rf_scene_set_attributes": lambda: L.rf_scene_set_attributes(None, None, None, 0),
        "rf_scene_update_positions": lambda: L.rf_scene_update_positions(None, None, None),
        "rf_scene_info": lambda: L.rf_scene_info(None, ctypes.byref(n64), ctypes.byref(e64), None, None),
        "rf_render_bwd": lambda: L.rf_render_bwd(None, cam, 1, ctypes.byref(opts), None, None, None, None,
                                                 None, None, None, None, None, None),
        "rf_render_bwd_ex": lambda: L.rf_render_bwd_ex(None, cam, 1, ctypes.byref(opts), None, None, None),
        "rf_trace_cells": lambda: L.rf_trace_cells(None, cam, ctypes.byref(opts), 4, None, None, None),
        "rf_mse_grad": lambda: L.rf_mse_grad(None, None, 3, 1.0, None, None, None),
        "rf_adjacency_create": lambda: L.rf_adjacency_create(None),
        "rf_adjacency_build": lambda: L.rf_adjacency_build(None, 10, None, None, 0, None),
        "rf_adjacency_result": lambda: L.rf_adjacency_result(None, None, None, None),
        "rf_adjacency_copy": lambda: L.rf_adjacency_copy(None, None, None, None),
        "rf_serve_create": lambda: L.rf_serve_create(None, None, None),
        "rf_serve_submit": lambda: L.rf_serve_submit(None, cam, None),
        "rf_serve_poll": lambda: L.rf_serve_poll(None, 0, None, None, None),
        "rf_serve_wait": lambda: L.rf_serve_wait(None, 0, 0, None, None),
        "rf_serve_stats": lambda: L.rf_serve_stats(None, None),
        "rf_serve_reset_stats": lambda: L.rf_serve_reset_stats(None),
        "rf_densify_scores": lambda: L.rf_densify_scores(None, None, None, None),
        "rf_prune_mask": lambda: L.rf_prune_mask(None, 0.1, None, None),
        "rf_sample_multinomial": lambda: L.rf_sample_multinomial(None, 4, None, 2, None, 0, None, None),
        "rf_render_fwd_noalloc": lambda: L.rf_render_fwd_noalloc(0, 0, None, None, None, None, None, 0, 0, None,
                                                                 cam, 1, ctypes.byref(opts), None, None, None,
                                                                 None),
    }
    for name, call in calls.items():
        assert call() == INVALID, name
        assert L.rf_last_error(), name
    # nothing to do: a zero-length loss and zero-size workspaces
    assert L.rf_mse_grad(None, None, 0, 1.0, None, None, None) == INVALID   # pointers still required
    assert L.rf_multinomial_workspace_bytes(0) == 0
    for destroy in ("rf_scene_destroy", "rf_adjacency_destroy", "rf_serve_destroy"):
        assert getattr(L, destroy)(None) == 0, destroy
