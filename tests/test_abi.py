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
    wb = cc.cicero_backward_workspace_size(_grid(), R, sp)
    assert wb > ws
    # with the weight gradients' operands: 2,272 bytes of split-BF16 rows per sample slot (R * 64 here)
    assert cc.cicero_backward_mlp_workspace_size(_grid(), R, sp) >= wb + 2272 * R * 64
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
    # record capacity: 2^24 rays x 256 slots reach 2^32 records unless max_records caps them
    sp256 = cc.sampling(n_samples=256)
    assert L.cicero_render_workspace_size(C.byref(_grid()), 1 << 24, C.byref(sp256), None) == 0
    assert b"2^32" in L.cicero_last_error()
    capped = cc.options(0, 8, max_records=100_000_000)
    assert L.cicero_render_workspace_size(C.byref(_grid()), 1 << 24, C.byref(sp256), C.byref(capped)) > 0
    # MLP tiles in flight per SM: 0 (as many as fit) .. 4
    for groups, ok in ((0, True), (4, True), (5, False), (-1, False)):
        size = L.cicero_render_workspace_size(C.byref(_grid()), 64, C.byref(sp), C.byref(cc.options(1, 4, 0, groups)))
        assert (size > 0) == ok, groups


def _mlp_desc(cc, in_dim=39, n_freq=4):
    m = cc.Mlp()
    m.in_dim, m.hidden, m.n_freq = in_dim, 128, n_freq
    m.w1 = m.b1 = m.w2 = m.b2 = m.w3 = m.b3 = 256
    return m


def test_batch_plan_validated_on_host(cc):
    L = cc.lib()
    keep = []

    def job(grid, n_samples=64, w=32, h=24):
        sp, cam, m = cc.sampling(n_samples=n_samples), cc.camera(w, h, 30.0, w / 2, h / 2, np.eye(3, 4)), _mlp_desc(cc)
        keep.extend([grid, sp, cam, m])
        j = cc.Job()
        j.grid, j.mlp, j.cam, j.sampling = C.addressof(grid), C.addressof(m), C.addressof(cam), C.addressof(sp)
        j.rgb, j.depth = 256, None
        return j

    arr = (cc.Job * 3)(job(_grid(dtype=1)), job(_grid(n=(96, 96, 96), dtype=1), 128, 40, 40),
                       job(_grid(n=(48, 48, 48), dtype=1), 32))
    bf16 = cc.options(cc.MLP_BF16, 8)
    size = L.cicero_batch_workspace_size(arr, 3, C.byref(bf16))
    table = L.cicero_batch_table_bytes(3)
    assert table >= 3 * 128 and table % 256 == 0
    rays = 32 * 24 * 2 + 40 * 40
    records = 32 * 24 * (64 + 32) + 40 * 40 * 128
    assert size > table + records * 52 + rays * 28  # table + per-record payload + per-ray headers
    # only the BF16 tensor-core path is batched
    assert L.cicero_batch_workspace_size(arr, 3, C.byref(cc.options(cc.MLP_FP32, 8))) == 0
    # jobs must share the grid dtype
    mixed = (cc.Job * 2)(job(_grid(dtype=1)), job(_grid(dtype=0)))
    assert L.cicero_batch_workspace_size(mixed, 2, C.byref(bf16)) == 0
    # job counts
    assert L.cicero_batch_workspace_size(arr, 0, C.byref(bf16)) == 0
    assert L.cicero_batch_table_bytes(0) == 0 and L.cicero_batch_table_bytes(2049) == 0
    # create rejects before touching the GPU
    h = C.c_void_p()
    st = L.cicero_batch_create(arr, 3, C.byref(cc.options(cc.MLP_FP32, 8)), C.c_void_p(1 << 20), size, C.byref(h))
    assert st == cc.ERR_UNSUPPORTED and not h.value
    st = L.cicero_batch_create(arr, 3, C.byref(bf16), C.c_void_p((1 << 20) + 8), size, C.byref(h))
    assert st == cc.ERR_INVALID_ARG  # workspace not 256-byte aligned
    assert L.cicero_batch_launch(None, None) == cc.ERR_INVALID_ARG


def test_extrapolate_pose_matches_oracle(cc):
    """Eq. 5-6 on the host side of the library (quaternions) against the oracle's axis-angle form."""
    import oracle
    import scenes
    cam = scenes.orbit_camera(64, 48)
    for (ka, kb, yaw, shift) in ((0, 1, 1.0, 0.005), (3, 4, -2.5, 0.02), (5, 6, 0.0, 0.01), (2, 3, 7.0, 0.0)):
        a, b = scenes.offset_camera(cam, ka, yaw, shift), scenes.offset_camera(cam, kb, yaw, shift)
        for lead in (0.0, 3.0, 10.5, 15.0, -1.0):
            got = cc.cicero_extrapolate_pose(cc.camera_from(a), cc.camera_from(b), lead)
            want = oracle.extrapolate_pose(a.c2w, b.c2w, lead)
            np.testing.assert_allclose(np.array(got.c2w[:]).reshape(3, 4), want, atol=3e-6)
            assert (got.width, got.height, got.f) == (b.width, b.height, np.float32(b.f))
    with pytest.raises(cc.CiceroError):
        cc.cicero_extrapolate_pose(cc.camera_from(cam), cc.camera_from(cam), float("nan"))


@pytest.mark.parametrize("lead", ["centred", "paper"])
@pytest.mark.parametrize("window,n_frames", [(4, 10), (3, 3), (16, 120), (6, 1)])
def test_reference_poses_follow_the_oracle_schedule(cc, orc, lead, window, n_frames):
    """cicero_reference_poses (host code of the library) against the oracle's schedule and FP64
    extrapolation.  The FP32 poses are orthonormal to ~1e-7 only, and the two sides take the
    rotation between them differently (the library by quaternion, the oracle by the trace and the
    skew part, whose angle is ill-conditioned for the small per-frame rotations), so the angle
    differs by a few 1e-7 rad and that difference is carried `lead` times: the tolerance grows with
    the lead (1e-5 rad at a lead of 24 frames is 0.01 pixel at f = 1100)."""
    import scenes
    cam = scenes.orbit_camera(64, 48)
    traj = [scenes.offset_camera(cam, k, yaw_deg=1.5, shift=0.01) for k in range(n_frames)]
    refs = cc.cicero_reference_poses([cc.camera_from(t) for t in traj], window, lead)
    sched = orc.reference_schedule(n_frames, window, lead)
    assert len(refs) == len(sched)
    for r, e in zip(refs, sched):
        got = np.array(r.c2w[:], np.float64).reshape(3, 4)
        want = traj[0].c2w.astype(np.float64) if e is None else orc.extrapolate_pose(traj[e[0]].c2w, traj[e[1]].c2w, e[2])
        np.testing.assert_allclose(got, want, atol=1e-6 + 5e-7 * (0.0 if e is None else e[2]))
        assert (r.width, r.height, r.f, r.cx, r.cy) == (cam.width, cam.height, np.float32(cam.f), cam.cx, cam.cy)
