"""CPU checks of the C ABI: the library loads, exports every entry point that include/cicero.h
declares, and rejects bad arguments on the host before touching the GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cc():
    from paper_2404_11852_gb300 import build, cicero
    build.build()
    cicero.lib()
    return cicero


def declared():
    txt = open(os.path.join(ROOT, "include", "cicero.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cicero_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(cc):
    names = declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", cc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (cicero_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(cc.lib(), n)


def test_version(cc):
    assert "sm_103a" in cc.cicero_version()


def _grid(n=(64, 64, 64), C_=12, dtype=0, feat=256):
    g = __import__("paper_2404_11852_gb300.cicero", fromlist=["Grid"]).Grid()
    g.n[:] = list(n)
    g.C = C_
    g.aabb_min[:] = [-1, -1, -1]
    g.aabb_max[:] = [1, 1, 1]
    g.act_shift = -4.0
    g.dtype = dtype
    g.density = 256
    g.features = feat
    return g


def test_workspace_size_queries(cc):
    sp = cc.sampling(n_samples=64)
    R = 64 * 64
    ws = cc.cicero_render_workspace_size(_grid(), R, sp)
    # at least the per-sample records (t, w, brick, sorted id: 4 B each; colour 16 B) of R*S slots
    assert ws >= R * 64 * 32
    assert cc.cicero_render_workspace_size(_grid(), R, sp, cc.options(1, 4)) > 0
    assert cc.cicero_backward_workspace_size(_grid(), R, sp) > ws
    cam = cc.camera(800, 800, 1000.0, 400.0, 400.0, np.eye(3, 4))
    assert cc.cicero_warp_workspace_size(cam) >= 800 * 800 * 8
    assert cc.cicero_mlp_eval_workspace_size(1000) >= 256


def test_invalid_arguments_rejected_on_host(cc):
    L = cc.lib()
    sp = cc.sampling(n_samples=64)
    cam = cc.camera(8, 8, 10.0, 4.0, 4.0, np.eye(3, 4))
    mlp = cc.Mlp()
    # NULL grid
    st = L.cicero_render(None, C.byref(mlp), C.byref(cam), C.byref(sp), None, None, None, None, None, None, 0, None)
    assert st == cc.ERR_INVALID_ARG
    assert b"grid" in L.cicero_last_error()
    # misaligned features (TMA needs 16-byte aligned rows)
    st = L.cicero_render(C.byref(_grid(feat=264)), C.byref(mlp), C.byref(cam), C.byref(sp), None, None, None, None,
                         None, None, 0, None)
    assert st == cc.ERR_ALIGNMENT
    # a row of n0 * C elements that is not a multiple of 16 bytes
    assert L.cicero_render_workspace_size(C.byref(_grid(n=(63, 64, 64), C_=3)), 64, C.byref(sp), None) == 0
    # too many channels for the MLP input
    assert L.cicero_render_workspace_size(C.byref(_grid(C_=24)), 64, C.byref(sp), None) == 0
    # bad sampling
    bad = cc.sampling(n_samples=0)
    assert L.cicero_render_workspace_size(C.byref(_grid()), 64, C.byref(bad), None) == 0
    # a camera with a non-finite pose
    badcam = cc.camera(8, 8, 10.0, 4.0, 4.0, np.full((3, 4), np.nan))
    st = L.cicero_warp(None, None, C.byref(badcam), C.byref(cam), 180.0, None, None, None, None, None, None, None,
                       None, 0, None)
    assert st == cc.ERR_INVALID_ARG
    # unsupported brick size
    st = L.cicero_render_workspace_size(C.byref(_grid()), 64, C.byref(sp), C.byref(cc.options(0, 5)))
    assert st == 0
