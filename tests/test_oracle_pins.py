"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes the oracle to something other than itself: a value that the mathematics
gives in closed form, an exact property (interpolation at vertices, exactness on affine
fields, identity warp), or an independent brute-force search.  A dropped term, a wrong
sign, a transposed axis or a wrong index in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import scenes

SIN = {1: 0.8414709848078965, 2: 0.9092974268256817, 4: -0.7568024953079282, 8: 0.9893582466233818}
COS = {1: 0.5403023058681398, 2: -0.4161468365471424, 4: -0.6536436208636119, 8: -0.14550003380861354}


def _const_grid(N, C, raw0, seed=3):
    dens = np.full((N, N, N), raw0, dtype=np.float64)
    feat = scenes.uniform(seed, N ** 3 * C, -1, 1).reshape(N, N, N, C)
    return scenes.Grid((N, N, N), C, dens, feat)


def _const_colour_mlp(C, b3):
    m = scenes.make_mlp(C, seed=7, random_bias=True)
    m.w3 = np.zeros_like(m.w3)
    m.b3 = np.asarray(b3, dtype=np.float32)
    return m


def _x_rays(n, x0=-0.9):
    yz = scenes.uniform(11, 2 * n, -0.5, 0.5).reshape(n, 2)
    o = np.stack([np.full(n, x0), yz[:, 0], yz[:, 1]], axis=1).astype(np.float32)
    d = np.tile(np.array([[1.0, 0.0, 0.0]], dtype=np.float32), (n, 1))
    return o, d


def _softplus(x):
    return math.log1p(math.exp(x))


# ---------------------------------------------------------------------------------------------
# camera rays (Sec. II-B Indexing: one ray per pixel; the pinhole of Eq. 1 and Eq. 3)


def _rotation(seed):
    """A seeded proper rotation (QR of a Gaussian matrix), rounded to FP32 like every pose."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q.astype(np.float32)


def _posed_camera(W, H, f, cx, cy, seed):
    c2w = np.concatenate([_rotation(seed), np.array([[0.3], [-1.2], [0.7]], np.float32)], axis=1)
    f32 = lambda v: float(np.float32(v))  # intrinsics are FP32 in every camera descriptor
    return scenes.Camera(W, H, f32(f), f32(cx), f32(cy), c2w)


@pytest.mark.parametrize("W,H", [(5, 3), (9, 15), (801, 799)])
def test_centre_pixel_looks_along_the_optical_axis(orc, W, H):
    """With the principal point at the image centre and odd sizes, the centre pixel's ray is the
    camera's z axis: column 2 of the rotation of c2w; every ray starts at column 3."""
    cam = _posed_camera(W, H, 0.9 * W, W / 2.0, H / 2.0, seed=W)
    p = (H // 2) * W + W // 2
    r = orc.camera_rays(cam, pix=np.array([p, 0], np.int32))
    R = cam.c2w.astype(np.float64)
    axis = R[:, 2] / np.linalg.norm(R[:, 2])
    np.testing.assert_allclose(r["d64"][0], axis, atol=1e-15)
    np.testing.assert_allclose(r["d32"][0], axis, atol=1e-7)
    np.testing.assert_array_equal(r["o64"], np.tile(R[:, 3], (2, 1)))
    assert not np.allclose(r["d64"][1], axis, atol=1e-3)  # a corner pixel looks elsewhere


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rays_project_back_to_their_pixel_centres(orc, seed):
    """Eq. 3 inverts the ray generation: a point on the ray of pixel p = j W + i, taken to camera
    space by the inverse of c2w and projected with u = f X / Z + cx, v = f Y / Z + cy, lands on
    the pixel centre (i + 1/2, j + 1/2).  Non-square, off-centre intrinsics and a general
    rotation, so a transposed rotation, swapped pixel axes or a missing half-pixel fail."""
    W, H = 7, 4
    cam = _posed_camera(W, H, 5.3 + seed, 2.9 - 0.4 * seed, 1.7 + 0.3 * seed, seed=10 + seed)
    r = orc.camera_rays(cam)
    M = cam.c2w.astype(np.float64)
    for rays_o, rays_d, tol in ((r["o64"], r["d64"], 1e-11), (r["o32"], r["d32"], 2e-5)):
        np.testing.assert_allclose(np.linalg.norm(rays_d, axis=1), 1.0, atol=1e-7)
        P = rays_o.astype(np.float64) + 2.7 * rays_d.astype(np.float64)
        Xc = np.linalg.solve(M[:, :3], (P - M[:, 3]).T).T
        assert (Xc[:, 2] > 0).all()
        u = cam.f * Xc[:, 0] / Xc[:, 2] + cam.cx
        v = cam.f * Xc[:, 1] / Xc[:, 2] + cam.cy
        i, j = np.arange(W * H) % W, np.arange(W * H) // W
        np.testing.assert_allclose(u, i + 0.5, atol=tol)
        np.testing.assert_allclose(v, j + 0.5, atol=tol)


def test_camera_axes_are_opencv(orc):
    """Identity pose: x to the right, y down, z forward; pixel lists select pixels p = j W + i."""
    W, H = 6, 4
    c2w = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    cam = scenes.Camera(W, H, 3.0, W / 2.0, H / 2.0, c2w)
    d = orc.camera_rays(cam)["d64"]
    i, j = np.arange(W * H) % W, np.arange(W * H) // W
    assert (np.sign(d[:, 0]) == np.sign(i + 0.5 - W / 2.0)).all()
    assert (np.sign(d[:, 1]) == np.sign(j + 0.5 - H / 2.0)).all()
    assert (d[:, 2] > 0).all()
    pick = np.array([13, 2, 23], np.int32)
    np.testing.assert_array_equal(orc.camera_rays(cam, pix=pick)["d64"], d[pick])


def test_orbit_camera_centre_ray_meets_the_look_at_point(orc):
    """The benchmark's orbit camera looks at the origin: the centre ray of an odd-sized image
    passes through it at distance |o|."""
    cam = scenes.orbit_camera(801, 801)
    r = orc.camera_rays(cam, pix=np.array([400 * 801 + 400], np.int32))
    o, d = r["o64"][0], r["d64"][0]
    np.testing.assert_allclose(o + np.linalg.norm(o) * d, 0.0, atol=1e-6)


# ---------------------------------------------------------------------------------------------
# accumulation (Sec. II-B) against the closed form of a homogeneous medium


def test_constant_density_closed_form(orc):
    raw0, S, L = 4.5, 32, 1.8
    g = _const_grid(8, 3, raw0)
    b3 = [0.3, -0.2, 1.0]
    m = _const_colour_mlp(3, b3)
    bg = (0.1, 0.2, 0.3)
    sp = scenes.Sampling(near=0.0, far=L, n_samples=S, t_stop=0.0, bg=bg)
    out = orc.render(g, m, sp, rays=_x_rays(16))
    sigma = _softplus(raw0 - 4.0)
    delta = np.float64(np.float32(L)) / S
    q = math.exp(-sigma * delta)
    acc = 1.0 - q ** S
    col = 1.0 / (1.0 + np.exp(-np.asarray(b3, dtype=np.float32).astype(np.float64)))
    rgb = col * acc + np.asarray(bg, dtype=np.float32).astype(np.float64) * (1.0 - acc)
    # sum_k q^k (1 - q) (near + (k + 1/2) delta) in closed form
    sk = q * (1 - S * q ** (S - 1) + (S - 1) * q ** S) / (1 - q) ** 2
    depth = ((1 - q) * (0.5 * delta * (1 - q ** S) / (1 - q) + delta * sk)) / acc
    np.testing.assert_allclose(out["acc"], acc, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["rgb"], np.tile(rgb, (16, 1)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["depth"], depth, rtol=1e-12)
    assert (out["n_steps"] == S).all() and not out["amb"].any()


def test_early_stop_closed_form(orc):
    raw0, S, L, t_stop = 8.0, 64, 1.8, 1e-3
    g = _const_grid(8, 2, raw0)
    m = _const_colour_mlp(2, [0.0, 0.0, 0.0])
    sp = scenes.Sampling(near=0.0, far=L, n_samples=S, t_stop=t_stop)
    out = orc.render(g, m, sp, rays=_x_rays(4))
    q = math.exp(-_softplus(raw0 - 4.0) * np.float64(np.float32(L)) / S)
    kstar = next(k for k in range(S + 1) if q ** k < np.float32(t_stop))
    assert (out["n_steps"] == kstar).all()
    np.testing.assert_allclose(out["acc"], 1 - q ** kstar, atol=1e-13)
    np.testing.assert_allclose(out["rgb"], 0.5 * (1 - q ** kstar), atol=1e-13)


def test_ambiguous_stop_returns_both_outcomes(orc):
    # sigma * delta = 1 per slot; t_stop placed on T_3 = e^-3 makes the decision before slot 3
    # ambiguous: the two outcomes differ by exactly the slot-3 weight T_3 (1 - e^-1).
    S, L = 16, 1.6
    delta = np.float64(np.float32(L)) / S
    sigma = 1.0 / delta
    raw0 = math.log(math.expm1(sigma)) + 4.0
    g = _const_grid(8, 2, raw0)
    m = _const_colour_mlp(2, [0.0, 0.0, 0.0])
    q = math.exp(-sigma * delta)
    sp = scenes.Sampling(near=0.0, far=L, n_samples=S, t_stop=float(np.float32(q ** 3)))
    out = orc.render(g, m, sp, rays=_x_rays(2))
    assert out["amb"].all()
    assert sorted({int(out["n_steps"][0]), int(out["n_steps_alt"][0])}) == [3, 4]
    np.testing.assert_allclose(np.abs(out["acc"] - out["acc_alt"]), q ** 3 * (1 - q), rtol=1e-6)


def test_affine_density_along_axis(orc):
    # raw(p) = a + b x: interpolation is exact, so sigma at slot k is softplus(a + b x_k - 4)
    N, S, L = 9, 40, 1.8
    a, b = 3.0, 2.0
    cb = np.zeros((2, 3))
    cb[0, 0] = b
    g = scenes.affine_grid(N, 1, np.array([a, 0.0]), cb)
    m = _const_colour_mlp(1, [0.0, 0.0, 0.0])
    sp = scenes.Sampling(near=0.0, far=L, n_samples=S, t_stop=0.0)
    out = orc.render(g, m, sp, rays=_x_rays(3))
    delta = np.float64(np.float32(L)) / S
    xk = np.float64(np.float32(-0.9)) + (np.arange(S) + 0.5) * delta
    tau = sum(_softplus(a + b * x - 4.0) for x in xk) * delta
    np.testing.assert_allclose(out["acc"], 1 - math.exp(-tau), rtol=1e-12)


def test_weights_invariants(orc):
    g = scenes.scene_small()
    m = scenes.make_mlp(12)
    cam = scenes.orbit_camera(24, 24, sampling=scenes.Sampling(bg=(1.0, 1.0, 1.0)))
    out = orc.render(g, m, cam.sampling, cam=cam)
    assert (out["acc"] >= 0).all() and (out["acc"] <= 1 + 1e-12).all()
    assert (out["rgb"] >= 0).all() and (out["rgb"] <= 1 + 1e-12).all()
    fin = np.isfinite(out["depth"])
    assert (out["acc"][fin] >= 0.5).all() and (out["acc"][~fin] < 0.5).all()
    # depth is a weighted mean of slot distances: inside [near, far]
    assert (out["depth"][fin] >= 0.5).all() and (out["depth"][fin] <= 2.5).all()


def test_black_background_white_scene_consistency(orc):
    # rgb with background b is rgb(bg=0) + T_end * b, and T_end = 1 - acc when no stop fires
    g = scenes.scene_small()
    m = scenes.make_mlp(12)
    cam = scenes.orbit_camera(16, 16)
    s0 = scenes.Sampling(t_stop=0.0)
    s1 = scenes.Sampling(t_stop=0.0, bg=(0.25, 0.5, 1.0))
    o0 = orc.render(g, m, s0, cam=cam)
    o1 = orc.render(g, m, s1, cam=cam)
    np.testing.assert_allclose(o1["rgb"], o0["rgb"] + (1 - o0["acc"])[:, None] * np.array([0.25, 0.5, 1.0]),
                               atol=1e-12)


# ---------------------------------------------------------------------------------------------
# Feature Gathering: trilinear interpolation


def test_trilinear_exact_on_affine_fields(orc):
    C = 5
    a = scenes.uniform(21, C + 1, -2, 2)
    b = scenes.uniform(22, 3 * (C + 1), -2, 2).reshape(C + 1, 3)
    g = scenes.affine_grid(11, C, a, b)
    p = scenes.uniform(23, 600, -1, 1).reshape(200, 3)
    raw, feat = orc.sample_grid(g, p)
    np.testing.assert_allclose(raw, a[0] + p @ b[0], atol=1e-13)
    np.testing.assert_allclose(feat, a[1:] + p @ b[1:].T, atol=1e-13)


def test_trilinear_reproduces_vertex_values(orc):
    N, C = 7, 3
    dens = scenes.uniform(31, N ** 3, -1, 1).reshape(N, N, N)
    feat = scenes.uniform(32, N ** 3 * C, -1, 1).reshape(N, N, N, C)
    g = scenes.Grid((N, N, N), C, dens, feat)
    idx = (scenes.splitmix64(33, 3 * 50) % np.uint64(N)).astype(int).reshape(50, 3)  # (x, y, z)
    p = -1.0 + 2.0 * idx / (N - 1)
    raw, f = orc.sample_grid(g, p)
    np.testing.assert_allclose(raw, dens[idx[:, 2], idx[:, 1], idx[:, 0]], atol=1e-14)
    np.testing.assert_allclose(f, feat[idx[:, 2], idx[:, 1], idx[:, 0]], atol=1e-14)


def test_trilinear_single_voxel_brute_force(orc):
    v = scenes.uniform(41, 8, -3, 3).reshape(2, 2, 2)
    g = scenes.Grid((2, 2, 2), 1, v.copy(), v[..., None].copy())
    p = scenes.uniform(42, 60, -1, 1).reshape(20, 3)
    f = (p + 1) / 2
    want = np.zeros(20)
    for z in range(2):
        for y in range(2):
            for x in range(2):
                wx = f[:, 0] if x else 1 - f[:, 0]
                wy = f[:, 1] if y else 1 - f[:, 1]
                wz = f[:, 2] if z else 1 - f[:, 2]
                want += wx * wy * wz * v[z, y, x]
    raw, feat = orc.sample_grid(g, p)
    np.testing.assert_allclose(raw, want, atol=1e-13)
    np.testing.assert_allclose(feat[:, 0], want, atol=1e-13)


# ---------------------------------------------------------------------------------------------
# Feature Computation: encoding and MLP


@pytest.mark.parametrize("axis,sign", [(0, 1), (1, 1), (2, 1), (0, -1), (2, -1)])
def test_positional_encoding_at_axes(orc, axis, sign):
    C = 2
    m = scenes.make_mlp(C)
    d = np.zeros((1, 3))
    d[0, axis] = sign
    x = orc.encode(m, np.array([[0.25, -0.5]]), d)[0]
    assert x.shape == (C + 27,)
    np.testing.assert_array_equal(x[:C], [0.25, -0.5])
    np.testing.assert_array_equal(x[C:C + 3], d[0])
    for k in range(4):
        s, c = x[C + 3 + 6 * k: C + 6 + 6 * k], x[C + 6 + 6 * k: C + 9 + 6 * k]
        want_s = np.zeros(3)
        want_s[axis] = sign * SIN[2 ** k]
        want_c = np.ones(3)
        want_c[axis] = COS[2 ** k]
        np.testing.assert_allclose(s, want_s, atol=1e-15)
        np.testing.assert_allclose(c, want_c, atol=1e-15)


def test_mlp_identity_weights(orc):
    C = 12
    m = scenes.make_mlp(C)
    I, H = m.in_dim, m.hidden
    m.w1 = np.zeros((H, I), dtype=np.float32)
    m.w1[np.arange(I), np.arange(I)] = 1
    m.w2 = np.eye(H, dtype=np.float32)
    m.w3 = np.zeros((3, H), dtype=np.float32)
    m.w3[[0, 1, 2], [0, 1, 2]] = 1
    x = scenes.uniform(51, 10 * I, -2, 2).reshape(10, I)
    c = orc.mlp_eval(m, x)
    np.testing.assert_allclose(c, 1 / (1 + np.exp(-np.maximum(x[:, :3], 0))), atol=1e-15)


def test_mlp_bias_only_output(orc):
    m = scenes.make_mlp(12, random_bias=True)
    m.w3 = np.zeros_like(m.w3)
    x = scenes.uniform(52, 5 * m.in_dim, -2, 2).reshape(5, m.in_dim)
    c = orc.mlp_eval(m, x)
    np.testing.assert_allclose(c, np.tile(1 / (1 + np.exp(-m.b3.astype(np.float64))), (5, 1)), atol=1e-15)


def test_mlp_single_hidden_unit_closed_form(orc):
    # only hidden unit j of both layers is live: c = sigmoid(w3 * relu(w2 * relu(w1 . x + b1) + b2) + b3)
    m = scenes.make_mlp(4)
    I, H = m.in_dim, m.hidden
    w1 = np.zeros((H, I), dtype=np.float32)
    w1[5] = scenes.uniform(53, I, -1, 1)
    w2 = np.zeros((H, H), dtype=np.float32)
    w2[9, 5] = 1.5
    w3 = np.zeros((3, H), dtype=np.float32)
    w3[:, 9] = [1.0, -2.0, 0.5]
    m.w1, m.w2, m.w3 = w1, w2, w3
    m.b1 = np.zeros(H, dtype=np.float32)
    m.b1[5] = 0.25
    m.b2 = np.zeros(H, dtype=np.float32)
    m.b3 = np.array([0.1, 0.2, 0.3], dtype=np.float32)
    x = scenes.uniform(54, 8 * I, -1, 1).reshape(8, I)
    h = np.maximum(1.5 * np.maximum(x @ w1[5].astype(np.float64) + 0.25, 0), 0)
    want = 1 / (1 + np.exp(-(h[:, None] * np.array([1.0, -2.0, 0.5]) + np.array([0.1, 0.2, 0.3], dtype=np.float32))))
    np.testing.assert_allclose(orc.mlp_eval(m, x), want, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# Indexing: which samples reach Feature Gathering and their bricks


def test_active_samples_axis_ray(orc):
    N, B, S, L = 33, 8, 48, 1.8
    g = _const_grid(N, 2, 0.0)
    sp = scenes.Sampling(near=0.0, far=L, n_samples=S, t_stop=0.0)
    o = np.array([[-0.9, 0.1, -0.3]], dtype=np.float32)
    d = np.array([[1.0, 0.0, 0.0]], dtype=np.float32)
    a = orc.active_samples(g, sp, B, rays=(o, d))
    assert len(a["slot"]) == S and (a["slot"] == np.arange(S)).all()
    delta = np.float64(np.float32(L)) / S
    x = -0.9 + (np.arange(S) + 0.5) * delta
    gx = (x + 1) * (N - 1) / 2
    gy, gz = (0.1 + 1) * (N - 1) / 2, (-0.3 + 1) * (N - 1) / 2
    nb = (N - 2) // B + 1
    want = (int(gz) // B * nb + int(gy) // B) * nb + np.floor(gx).astype(int) // B
    safe = np.abs(gx - np.round(gx)) > 1e-4
    np.testing.assert_array_equal(a["brick"][safe], want[safe])
    # the voxel of each sample: floor of the vertex coordinate along x, fixed y and z
    want_v = (int(gz) * N + int(gy)) * N + np.floor(gx).astype(int)
    np.testing.assert_array_equal(a["voxel"][safe], want_v[safe])


def test_active_samples_respect_occupancy(orc):
    N, R = 17, 4
    g = _const_grid(N, 2, 0.0)
    occ = np.zeros((R, R, R), dtype=np.uint8)
    occ[:, :, 1] = 1  # only cells with x-cell index 1: x in [-0.5, 0)
    g.occ = occ
    sp = scenes.Sampling(near=0.0, far=1.8, n_samples=36, t_stop=0.0)
    o = np.array([[-0.9, 0.05, 0.05]], dtype=np.float32)
    d = np.array([[1.0, 0.0, 0.0]], dtype=np.float32)
    a = orc.active_samples(g, sp, 4, rays=(o, d))
    x = -0.9 + (a["slot"] + 0.5) * 0.05
    assert len(x) > 0 and (x >= -0.5 - 1e-6).all() and (x < 0.0 + 1e-6).all()
    assert len(x) == 10


def test_march_mode_slots_stay_in_box(orc):
    g = _const_grid(9, 2, 0.0)
    sp = scenes.Sampling(near=0.0, far=1e30, n_samples=1000, step=0.01, t_stop=0.0)
    o = np.array([[-3.0, 0.2, 0.1]], dtype=np.float32)
    d = np.array([[1.0, 0.0, 0.0]], dtype=np.float32)
    a = orc.active_samples(g, sp, 4, rays=(o, d))
    # entry at t = 2, exit at t = 4: slots 2 + (k + 1/2) 0.01 < 4  ->  k < 199.5
    assert len(a["slot"]) == 200 and a["slot"][-1] == 199


# ---------------------------------------------------------------------------------------------
# SpaRW (Sec. III-B): warp against identity, translation, rotation and brute force


def _fwd_cam(W, H, f, t=(0.0, 0.0, 0.0), R=None):
    c2w = np.zeros((3, 4), dtype=np.float32)
    c2w[:, :3] = np.eye(3) if R is None else R
    c2w[:, 3] = t
    return scenes.Camera(W, H, float(f), W / 2.0, H / 2.0, c2w)


def _plane_depth(cam, Z):
    j, i = np.mgrid[0:cam.height, 0:cam.width]
    dx = (i + 0.5 - cam.cx) / cam.f
    dy = (j + 0.5 - cam.cy) / cam.f
    return (Z * np.sqrt(dx * dx + dy * dy + 1.0)).astype(np.float32).ravel()


def test_identity_warp_is_exact_copy(orc):
    g = scenes.scene_small()
    cam = scenes.orbit_camera(32, 32)
    rgb = scenes.uniform(61, 32 * 32 * 3).astype(np.float32).reshape(-1, 3)
    depth = scenes.uniform(62, 32 * 32, 1.0, 2.0).astype(np.float32)
    depth[::7] = np.inf
    w = orc.warp(rgb, depth, cam, cam, void_grid=g, void_sampling=cam.sampling)
    assert w["n_holes"] == 0 and (w["mask"] == 0).all()
    np.testing.assert_array_equal(w["rgb"], rgb)
    np.testing.assert_array_equal(w["src"], np.arange(32 * 32))


def test_translation_shifts_by_f_t_over_Z(orc):
    W = H = 32
    ref = _fwd_cam(W, H, 16.0)
    tgt = _fwd_cam(W, H, 16.0, t=(0.25, 0.0, 0.0))
    depth = _plane_depth(ref, 2.0)  # shift = 16 * 0.25 / 2 = 2 px to the left
    rgb = scenes.uniform(63, W * H * 3).astype(np.float32).reshape(-1, 3)
    w = orc.warp(rgb, depth, ref, tgt)
    src = w["src"].reshape(H, W)
    j, i = np.mgrid[0:H, 0:W]
    np.testing.assert_array_equal(src[:, :W - 2], (j * W + i + 2)[:, :W - 2])
    assert (src[:, W - 2:] == -1).all()
    assert w["n_holes"] == 2 * H
    np.testing.assert_array_equal(w["rgb"].reshape(H, W, 3)[:, :W - 2], rgb.reshape(H, W, 3)[:, 2:])


def test_disocclusion_width_closed_form(orc):
    # foreground square at Z=1 over a background at Z=4; a 0.25 sideways step uncovers
    # f t (1/Z_fg - 1/Z_bg) = 16 * 0.25 * 0.75 = 3 columns behind the square, plus the 1-column
    # background edge.
    W = H = 32
    ref = _fwd_cam(W, H, 16.0)
    tgt = _fwd_cam(W, H, 16.0, t=(0.25, 0.0, 0.0))
    Z = np.full((H, W), 4.0)
    Z[8:24, 12:20] = 1.0
    j, i = np.mgrid[0:H, 0:W]
    dx, dy = (i + 0.5 - 16) / 16, (j + 0.5 - 16) / 16
    depth = (Z * np.sqrt(dx * dx + dy * dy + 1)).astype(np.float32).ravel()
    w = orc.warp(np.zeros((W * H, 3), np.float32), depth, ref, tgt)
    holes = (w["mask"].reshape(H, W) == 1)
    want = np.zeros((H, W), bool)
    want[8:24, 16:19] = True
    want[:, W - 1] = True
    np.testing.assert_array_equal(holes, want)


def test_rotation_of_points_at_infinity_is_homography(orc):
    W = H = 40
    f = 30.0
    th = math.radians(4.0)
    Ry = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    ref = _fwd_cam(W, H, f)
    tgt = _fwd_cam(W, H, f, R=Ry)
    depth = np.full(W * H, np.inf, dtype=np.float32)
    w = orc.warp(np.zeros((W * H, 3), np.float32), depth, ref, tgt)
    K = np.array([[f, 0, W / 2], [0, f, H / 2], [0, 0, 1]])
    Hm = K @ Ry.astype(np.float32).astype(np.float64).T @ np.linalg.inv(K)
    j, i = np.mgrid[0:H, 0:W]
    uv = np.stack([i.ravel() + 0.5, j.ravel() + 0.5, np.ones(W * H)])
    q = Hm @ uv
    u, v = q[0] / q[2], q[1] / q[2]
    inside = (u >= 0) & (u < W) & (v >= 0) & (v < H)
    near_edge = (np.abs(u - np.round(u)) < 1e-3) | (np.abs(v - np.round(v)) < 1e-3)
    want = np.full(W * H, -1)
    unsure = np.zeros(W * H, bool)
    for qi in np.nonzero(inside)[0][::-1]:  # lower index wins: write in descending order
        p = int(np.floor(v[qi])) * W + int(np.floor(u[qi]))
        want[p] = qi
    for qi in np.nonzero(near_edge)[0]:
        for du in (-1e-3, 1e-3):
            for dv in (-1e-3, 1e-3):
                uu, vv = u[qi] + du, v[qi] + dv
                if 0 <= uu < W and 0 <= vv < H:
                    unsure[int(np.floor(vv)) * W + int(np.floor(uu))] = True
    ok = ~unsure
    assert ok.sum() > 0.8 * W * H
    np.testing.assert_array_equal(w["src"][ok], want[ok])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_warp_depth_test_matches_brute_force(orc, seed):
    W = H = 16
    ref = scenes.orbit_camera(W, H)
    tgt = scenes.offset_camera(ref, 3 + seed, yaw_deg=1.5, shift=0.02)
    depth = scenes.uniform(70 + seed, W * H, 1.0, 2.5).astype(np.float32)
    depth[scenes.uniform(80 + seed, W * H) < 0.2] = np.inf
    w = orc.warp(np.zeros((W * H, 3), np.float32), depth, ref, tgt)
    bf = orc.warp_bruteforce(depth, ref, tgt)
    np.testing.assert_array_equal(w["src"], bf)
    assert (w["src"] >= 0).sum() > 0.5 * W * H


def test_warp_angle_threshold(orc):
    W = H = 16
    ref = _fwd_cam(W, H, 16.0)
    tgt = _fwd_cam(W, H, 16.0, t=(0.25, 0.0, 0.0))
    depth = _plane_depth(ref, 2.0)
    # angle at a point on the optical axis plane: atan(0.25 / 2) = 7.1 deg
    w_hi = orc.warp(np.zeros((W * H, 3), np.float32), depth, ref, tgt, max_angle_deg=10.0)
    w_lo = orc.warp(np.zeros((W * H, 3), np.float32), depth, ref, tgt, max_angle_deg=5.0)
    assert (w_hi["src"] >= 0).sum() > 0.8 * W * H
    assert (w_lo["src"] >= 0).sum() == 0


def test_relative_pose_composes_back(orc):
    ref = scenes.orbit_camera(8, 8)
    tgt = scenes.offset_camera(ref, 5)
    T = orc.rel_pose(ref, tgt).astype(np.float64)
    M = lambda c: np.vstack([c.c2w.astype(np.float64), [0, 0, 0, 1]])
    np.testing.assert_allclose(M(tgt) @ np.vstack([T, [0, 0, 0, 1]]), M(ref), atol=1e-6)


def test_void_holes(orc):
    g = scenes.scene_small()
    cam = scenes.orbit_camera(24, 24)
    tgt = scenes.offset_camera(cam, 8, yaw_deg=3.0)
    depth = np.full(24 * 24, np.inf, dtype=np.float32)
    depth[:24 * 12] = 1.2  # top half at finite depth, the rest void
    # holes whose ray misses the box get the background colour and are not listed
    far_box = scenes.Grid(g.n, g.C, g.density, g.features, (5.0, 5.0, 5.0), (6.0, 6.0, 6.0))
    w = orc.warp(np.zeros((576, 3), np.float32), depth, cam, tgt, void_grid=far_box,
                 void_sampling=scenes.Sampling(bg=(0.5, 0.5, 0.5)))
    holes = w["mask"] != 0
    assert holes.sum() > 0 and (w["mask"][holes] == 2).all() and w["n_holes"] == 0
    np.testing.assert_array_equal(w["rgb"][holes], 0.5)
    w2 = orc.warp(np.zeros((576, 3), np.float32), depth, cam, tgt, void_grid=g)
    assert w2["n_holes"] > 0
    assert (np.diff(w2["hole_idx"]) > 0).all()


# ---------------------------------------------------------------------------------------------
# gradients against FP64 central differences


def _fd_setup():
    g = scenes.scene_fd()
    m = scenes.make_mlp(4, random_bias=True)
    o, d = scenes.random_rays(32)
    tgt = scenes.random_targets(32).astype(np.float64)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=32, t_stop=0.0)
    return g, m, (o, d), tgt, sp


def _loss(orc, g, m, rays, tgt, sp):
    out = orc.render(g, m, sp, rays=rays)
    return float(np.mean((out["rgb"] - tgt) ** 2)), out


def _fd_check(orc, arr, idx, an, scale, g, m, rays, tgt, sp, L0, h=1e-6):
    """Central difference at arr.flat[idx]; a parameter whose +h and -h one-sided slopes
    disagree beyond smooth curvature crossed a ReLU kink and is skipped (returns None)."""
    orig = arr.flat[idx]
    arr.flat[idx] = orig + h
    Lp, _ = _loss(orc, g, m, rays, tgt, sp)
    arr.flat[idx] = orig - h
    Lm, _ = _loss(orc, g, m, rays, tgt, sp)
    arr.flat[idx] = orig
    if abs((Lp - L0) / h - (L0 - Lm) / h) > 1e-4 * scale:
        return None
    return (Lp - Lm) / (2 * h)


def test_gradient_matches_central_differences(orc):
    g, m, rays, tgt, sp = _fd_setup()
    L0, out = _loss(orc, g, m, rays, tgt, sp)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    dd, df, _ = orc.backward(g, m, sp, grad, rays=rays)
    worst, skipped, n = 0.0, 0, 0
    for arr, an in ((g.density, dd), (g.features, df)):
        flat = an.ravel()
        scale = np.abs(flat).max()
        assert scale > 0
        nz, z = np.nonzero(flat != 0)[0], np.nonzero(flat == 0)[0]
        picks = list(np.argsort(-np.abs(flat))[:15])
        picks += list(nz[(scenes.splitmix64(90, 10) % np.uint64(len(nz))).astype(int)])
        picks += list(z[(scenes.splitmix64(91, 5) % np.uint64(len(z))).astype(int)])
        for i in picks:
            fd = _fd_check(orc, arr, i, flat[i], scale, g, m, rays, tgt, sp, L0)
            n += 1
            if fd is None:
                skipped += 1
                continue
            worst = max(worst, abs(fd - flat[i]) / scale)
    assert skipped <= 0.1 * n, (skipped, n)
    assert worst <= 1e-6, worst


def test_mlp_gradient_matches_central_differences(orc):
    g, m, rays, tgt, sp = _fd_setup()
    m64 = scenes.Mlp(*[w.astype(np.float64) for w in (m.w1, m.b1, m.w2, m.b2, m.w3, m.b3)], m.n_freq)
    L0, out = _loss(orc, g, m64, rays, tgt, sp)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    _, _, dm = orc.backward(g, m64, sp, grad, rays=rays, with_mlp=True)
    names = ["w1", "b1", "w2", "b2", "w3", "b3"]
    off, worst, skipped, n = 0, 0.0, 0, 0
    scale = np.abs(dm).max()
    for nme in names:
        arr = getattr(m64, nme)
        k = arr.size
        sub = dm[off:off + k]
        for i in list(np.argsort(-np.abs(sub))[:4]) + [int(scenes.splitmix64(95, 1)[0] % np.uint64(k))]:
            fd = _fd_check(orc, arr, i, sub[i], scale, g, m64, rays, tgt, sp, L0)
            n += 1
            if fd is None:
                skipped += 1
                continue
            worst = max(worst, abs(fd - sub[i]) / scale)
        off += k
    assert off == dm.size
    assert skipped <= 0.2 * n, (skipped, n)
    assert worst <= 1e-6, worst


# ---------------------------------------------------------------------------------------------
# reference-pose extrapolation (Sec. III-C, Eq. 5-6)


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_extrapolate_translation_closed_form(orc):
    p1, p2 = np.array([0.1, -0.2, 1.5]), np.array([0.13, -0.18, 1.49])
    prev = np.concatenate([np.eye(3), p1[:, None]], 1)
    cur = np.concatenate([np.eye(3), p2[:, None]], 1)
    for lead in (0.5, 3.0, 10.5, 15.0):
        r = orc.extrapolate_pose(prev, cur, lead)
        np.testing.assert_allclose(r[:, 3], p2 + lead * (p2 - p1), atol=1e-15)  # Eq. 5-6
        np.testing.assert_allclose(r[:, :3], np.eye(3), atol=1e-15)


def test_extrapolate_rotation_about_fixed_axis(orc):
    th0, a = 0.3, np.radians(1.0)
    R1 = _rz(th0) @ _rz(0.1)  # any orientation, then turning about world z by a per frame
    R2 = _rz(a) @ R1
    prev = np.concatenate([R1, np.zeros((3, 1))], 1)
    cur = np.concatenate([R2, np.zeros((3, 1))], 1)
    for lead in (1.0, 8.0, 10.5):
        r = orc.extrapolate_pose(prev, cur, lead)
        np.testing.assert_allclose(r[:, :3], _rz(lead * a) @ R2, atol=1e-13)


def test_extrapolate_special_leads(orc):
    cam = scenes.orbit_camera(64, 64)
    t0, t1 = scenes.offset_camera(cam, 0).c2w, scenes.offset_camera(cam, 1, yaw_deg=2.0, shift=0.02).c2w
    np.testing.assert_allclose(orc.extrapolate_pose(t0, t1, 0.0), t1, atol=1e-12)   # no lead: the latest pose
    np.testing.assert_allclose(orc.extrapolate_pose(t0, t1, -1.0), t0, atol=1e-6)   # one frame back
    np.testing.assert_allclose(orc.extrapolate_pose(t1, t1, 7.0), t1, atol=1e-12)   # standing still


def test_extrapolate_trajectory_generator(orc):
    """The trajectory generator turns about a fixed axis and moves along a fixed direction at a
    constant rate, so extrapolating k frames ahead lands on frame k ahead (to float rounding)."""
    cam = scenes.orbit_camera(64, 64)
    t = [scenes.offset_camera(cam, k).c2w.astype(np.float64) for k in range(20)]
    for a, lead in ((1, 3), (4, 8), (9, 10)):
        np.testing.assert_allclose(orc.extrapolate_pose(t[a - 1], t[a], lead), t[a + lead], atol=2e-6)


# ---------------------------------------------------------------------------------------------
# bilinear resampling of the DS-2 comparator


def test_upsample_constant_identity_and_ramp(orc):
    img = np.full((5, 7, 3), 0.37)
    np.testing.assert_allclose(orc.upsample_bilinear(img, 14, 10), 0.37, atol=1e-15)
    rnd = np.random.default_rng(3).random((6, 9, 2))
    np.testing.assert_allclose(orc.upsample_bilinear(rnd, 9, 6), rnd, atol=1e-15)  # same size: identity
    # a ramp a + b x along x is reproduced at every output centre, clamped at the image edges
    w, W, a, b = 8, 20, 0.25, 0.1
    ramp = np.broadcast_to((a + b * np.arange(w))[None, :, None], (3, w, 1))
    out = orc.upsample_bilinear(ramp, W, 3)[0, :, 0]
    u = np.clip((np.arange(W) + 0.5) * w / W - 0.5, 0, w - 1)
    np.testing.assert_allclose(out, a + b * u, atol=1e-14)
    assert out[0] == a and out[-1] == a + b * (w - 1)


# ---------------------------------------------------------------------------------------------
# multiresolution hash encoding (the hash-grid workload)


def _hash_scene(levels=3, log2_size=10, res=(4, 8, 40), table=None):
    h = scenes.HashGrid(levels, 2, log2_size, tuple(res),
                        table if table is not None else np.zeros((levels, 1 << log2_size, 2), np.float32))
    return scenes.with_hash(scenes.scene_fd().astype(np.float32), h)


def test_hash_constant_table(orc):
    g = _hash_scene(table=np.full((3, 1024, 2), 0.625, np.float32))
    p = scenes.uniform(7, 60, -1.0, 1.0).reshape(20, 3)
    np.testing.assert_allclose(orc.hash_features(g, p), 0.625, atol=1e-15)


def test_hash_dense_level_is_exact_on_linear_fields(orc):
    """Level 0 (4 cells, 125 vertices <= 1024 entries) is stored densely at x + 5 (y + 5 z): a
    linear field written at its vertices is reproduced exactly anywhere in the box."""
    N, T = 4, 1024
    tab = np.zeros((3, T, 2), np.float32)
    for z in range(N + 1):
        for y in range(N + 1):
            for x in range(N + 1):
                tab[0, x + (N + 1) * (y + (N + 1) * z)] = [0.25 * x - 0.5 * y + 0.125 * z, 0.5 + 0.25 * z]
    g = _hash_scene(table=tab)
    p = scenes.uniform(8, 90, -1.0, 1.0).reshape(30, 3)
    v = (p + 1.0) / 2.0 * N  # vertex coordinates of level 0
    got = orc.hash_features(g, p)[:, :2]
    np.testing.assert_allclose(got[:, 0], 0.25 * v[:, 0] - 0.5 * v[:, 1] + 0.125 * v[:, 2], atol=1e-12)
    np.testing.assert_allclose(got[:, 1], 0.5 + 0.25 * v[:, 2], atol=1e-12)


def test_hash_vertices_on_the_x_axis(orc):
    """Level 2 (40 cells: 68921 vertices > 1024 entries) is hashed; on the x axis (y = z = 0) the
    spatial hash reduces to x mod T, and at a vertex the interpolation returns that one entry."""
    tab = (np.arange(3 * 1024 * 2, dtype=np.float32).reshape(3, 1024, 2) * 1e-3).astype(np.float32)
    g = _hash_scene(table=tab)
    for x in (0, 1, 17, 39):
        p = np.array([[-1.0 + 2.0 * x / 40.0, -1.0, -1.0]])
        np.testing.assert_allclose(orc.hash_features(g, p)[0, 4:6], tab[2, x % 1024], atol=1e-9)


def test_hash_continuous_across_cell_faces(orc):
    g = _hash_scene(table=scenes.uniform(9, 3 * 1024 * 2, -1.0, 1.0).astype(np.float32).reshape(3, 1024, 2))
    x_face = -1.0 + 2.0 * 7.0 / 40.0  # a face of level 2 (and of no coarser level)
    p = np.array([[x_face - 1e-9, 0.13, -0.41], [x_face + 1e-9, 0.13, -0.41]])
    f = orc.hash_features(g, p)
    np.testing.assert_allclose(f[0], f[1], atol=1e-7)


def test_extrapolate_paper_example_n4(orc):
    """The Eq. 6 example of Sec. III-C (tests/golden/eq6_reference_pose_n4.txt): lead N/2 = 2."""
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "eq6_reference_pose_n4.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = np.array([float(x) for x in v])
    prev = np.concatenate([np.eye(3), rows["T1"][:, None]], 1)
    cur = np.concatenate([np.eye(3), rows["T2"][:, None]], 1)
    r = orc.extrapolate_pose(prev, cur, rows["N"][0] / 2)
    np.testing.assert_array_equal(r[:, 3], rows["R1"])  # dyadic values: exact in FP64
    np.testing.assert_array_equal(r[:, :3], np.eye(3))


def test_reference_schedule_reproduces_the_paper_example(orc):
    """The Eq. 6 example of Sec. III-C through the schedule: with Eq. 6 read literally and windows
    of N = 4, the second reference is extrapolated from the first two frames (T1, T2) by N/2 = 2
    intervals, which gives R1 of tests/golden/eq6_reference_pose_n4.txt."""
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "eq6_reference_pose_n4.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = np.array([float(x) for x in v])
    N = int(rows["N"][0])
    sched = orc.reference_schedule(3 * N, N, lead="paper")
    assert sched[0] is None and len(sched) == 3
    prev, cur, lead = sched[1]
    assert (prev, cur, lead) == (0, 1, N / 2)
    poses = [np.concatenate([np.eye(3), rows[k][:, None]], 1) for k in ("T1", "T2")]
    r = orc.extrapolate_pose(poses[prev], poses[cur], lead)
    np.testing.assert_array_equal(r[:, 3], rows["R1"])


def test_reference_schedule_centres_each_reference(orc):
    """On a constant-velocity straight path the extrapolation is exact, so each reference lands on
    the centre of the window it serves (centred lead), or N/2 frames after the latest known pose
    (Eq. 6 literally), which is a window behind."""
    N, n = 4, 14
    pos = lambda t: np.array([0.1 * t, -0.05 * t, 0.02 * t])
    poses = [np.concatenate([np.eye(3), pos(i)[:, None]], 1) for i in range(n)]
    for lead, centre in (("centred", lambda w: w * N + N / 2.0), ("paper", lambda w: max(1, (w - 1) * N) + N / 2.0)):
        for w, e in enumerate(orc.reference_schedule(n, N, lead)):
            if e is None:
                continue
            r = orc.extrapolate_pose(poses[e[0]], poses[e[1]], e[2])
            np.testing.assert_allclose(r[:, 3], pos(centre(w)), atol=1e-12)
