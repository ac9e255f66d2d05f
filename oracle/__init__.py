"""Python access to the FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  The product package never imports it.

Inputs are the arrays of ``scenes`` (grids, MLP weights, cameras, rays); outputs are numpy
float64 arrays.  See ``oracle.c`` for the definitions and the paper passages they follow.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrGrid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("C", C.c_int), ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3),
                ("act_shift", C.c_double), ("dtype", C.c_int), ("density", C.c_void_p),
                ("features", C.c_void_p), ("occ", C.c_void_p), ("occ_res", C.c_int), ("hash", C.c_void_p)]


class OrHash(C.Structure):
    _fields_ = [("levels", C.c_int), ("feat", C.c_int), ("log2_size", C.c_int), ("res", C.c_int * 16),
                ("dtype", C.c_int), ("table", C.c_void_p)]


class OrMlp(C.Structure):
    _fields_ = [("in_dim", C.c_int), ("hidden", C.c_int), ("n_freq", C.c_int), ("dtype", C.c_int),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p)]


class OrSampling(C.Structure):
    _fields_ = [("near_t", C.c_float), ("far_t", C.c_float), ("n_samples", C.c_int), ("step", C.c_float),
                ("t_stop", C.c_float), ("bg", C.c_float * 3), ("void_acc", C.c_float)]


class OrRays(C.Structure):
    _fields_ = [("kind", C.c_int), ("width", C.c_int), ("height", C.c_int), ("f", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("c2w", C.c_float * 12), ("pix", C.c_void_p),
                ("n_pix", C.c_int), ("o", C.c_void_p), ("d", C.c_void_p), ("n_rays", C.c_int)]


class OrCam(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("f", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("c2w", C.c_float * 12)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_render.argtypes = [P] * 13 + [C.c_int]
        L.or_render.restype = C.c_int
        L.or_active_samples.argtypes = [P, P, P, C.c_int, P, P, P, P, C.c_long, P, P]
        L.or_active_samples.restype = C.c_long
        L.or_sample_grid.argtypes = [P, P, C.c_int, P, P]
        L.or_hash_features.argtypes = [P, P, C.c_int, P]
        L.or_mlp_eval.argtypes = [P, P, C.c_int, P]
        L.or_encode.argtypes = [P, C.c_int, P, P, C.c_int, P]
        L.or_warp.argtypes = [P, P, P, P, C.c_float, P, P, P, P, P, P, P, P]
        L.or_warp.restype = C.c_int
        L.or_warp_bruteforce.argtypes = [P, P, P, C.c_float, P]
        L.or_rel_pose.argtypes = [P, P, P]
        L.or_backward.argtypes = [P] * 8
        L.or_backward.restype = C.c_int
        L.or_relu_margin.argtypes = [P] * 5
        L.or_max_threads.restype = C.c_int
        L.or_rays_of.argtypes = [P] * 5
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def __call__(self, a):
        self.refs.append(a)
        return a


_DT = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.float16): 2}


def _grid(g, keep) -> OrGrid:
    dens = keep(np.ascontiguousarray(g.density))
    feat = keep(np.ascontiguousarray(g.features if g.features is not None else np.zeros(1, dens.dtype)))
    assert dens.dtype == feat.dtype
    s = OrGrid()
    s.n[:] = list(g.n)
    s.C = g.C
    s.aabb_min[:] = list(g.aabb_min)
    s.aabb_max[:] = list(g.aabb_max)
    s.act_shift = g.act_shift
    s.dtype = _DT[dens.dtype]
    s.density = dens.ctypes.data
    s.features = feat.ctypes.data
    if g.occ is not None:
        occ = keep(np.ascontiguousarray(g.occ, dtype=np.uint8))
        s.occ = occ.ctypes.data
        s.occ_res = occ.shape[0]
    h = getattr(g, "hash", None)
    if h is not None:
        hs = OrHash()
        hs.levels, hs.feat, hs.log2_size = h.levels, h.feat, h.log2_size
        hs.res[: h.levels] = list(h.res)
        tab = keep(np.ascontiguousarray(h.table))
        hs.dtype = 1 if tab.dtype == np.float32 else 2
        hs.table = tab.ctypes.data
        keep(hs)
        s.hash = C.addressof(hs)
    return s


def _mlp(m, keep) -> OrMlp:
    s = OrMlp()
    arrs = [keep(np.ascontiguousarray(a)) for a in (m.w1, m.b1, m.w2, m.b2, m.w3, m.b3)]
    s.in_dim, s.hidden, s.n_freq = m.in_dim, m.hidden, m.n_freq
    s.dtype = 0 if arrs[0].dtype == np.float64 else 1
    s.w1, s.b1, s.w2, s.b2, s.w3, s.b3 = [a.ctypes.data for a in arrs]
    return s


def _sampling(sp) -> OrSampling:
    s = OrSampling()
    s.near_t, s.far_t, s.n_samples, s.step, s.t_stop = sp.near, sp.far, sp.n_samples, sp.step, sp.t_stop
    s.bg[:] = list(sp.bg)
    s.void_acc = sp.void_acc
    return s


def _cam(cam) -> OrCam:
    s = OrCam()
    s.width, s.height, s.f, s.cx, s.cy = cam.width, cam.height, cam.f, cam.cx, cam.cy
    s.c2w[:] = [float(v) for v in np.asarray(cam.c2w, dtype=np.float32).ravel()]
    return s


def _camera_rays(cam, pix, keep) -> OrRays:
    s = OrRays()
    s.kind = 0
    s.width, s.height, s.f, s.cx, s.cy = cam.width, cam.height, cam.f, cam.cx, cam.cy
    s.c2w[:] = [float(v) for v in np.asarray(cam.c2w, dtype=np.float32).ravel()]
    if pix is not None:
        p = keep(np.ascontiguousarray(pix, dtype=np.int32))
        s.pix = p.ctypes.data
        s.n_pix = p.size
    return s


def _explicit_rays(o, d, keep) -> OrRays:
    s = OrRays()
    s.kind = 1
    o = keep(np.ascontiguousarray(o, dtype=np.float32))
    d = keep(np.ascontiguousarray(d, dtype=np.float32))
    s.o, s.d, s.n_rays = o.ctypes.data, d.ctypes.data, o.shape[0]
    return s


def _rays(keep, cam=None, pix=None, rays=None):
    if rays is not None:
        return _explicit_rays(rays[0], rays[1], keep)
    return _camera_rays(cam, pix, keep)


def _nrays(cam=None, pix=None, rays=None):
    if rays is not None:
        return int(np.asarray(rays[0]).shape[0])
    return int(len(pix)) if pix is not None else cam.width * cam.height


def render(grid, mlp, sampling, cam=None, pix=None, rays=None, threads: int = 0) -> dict:
    """Render the rays of ``cam`` (every pixel, or the pixels in ``pix``) or the explicit
    ``rays=(o, d)``.  Returns rgb [R,3], depth, acc, n_steps, amb and the *_alt outcome."""
    keep = _Keep()
    g, m, s = _grid(grid, keep), _mlp(mlp, keep), _sampling(sampling)
    r = _rays(keep, cam, pix, rays)
    R = _nrays(cam, pix, rays)
    out = {k: np.zeros((R, 3)) for k in ("rgb", "rgb_alt")}
    for k in ("depth", "acc", "depth_alt", "acc_alt"):
        out[k] = np.zeros(R)
    for k in ("n_steps", "amb", "n_steps_alt"):
        out[k] = np.zeros(R, dtype=np.int32)
    rc = lib().or_render(C.byref(g), C.byref(m), C.byref(r), C.byref(s), _ptr(out["rgb"]), _ptr(out["depth"]),
                         _ptr(out["acc"]), _ptr(out["n_steps"]), _ptr(out["amb"]), _ptr(out["rgb_alt"]),
                         _ptr(out["depth_alt"]), _ptr(out["acc_alt"]), _ptr(out["n_steps_alt"]), threads)
    if rc != 0:
        raise ValueError(f"or_render failed ({rc})")
    out["amb"] = out["amb"].astype(bool)
    return out


def active_samples(grid, sampling, brick: int, cam=None, pix=None, rays=None, cap: int | None = None) -> dict:
    """The samples that reach Feature Gathering with their brick id and voxel (FP32 decisions)."""
    keep = _Keep()
    g, s = _grid(grid, keep), _sampling(sampling)
    r = _rays(keep, cam, pix, rays)
    R = _nrays(cam, pix, rays)
    cap = cap or R * sampling.n_samples
    ray_of = np.zeros(cap, dtype=np.int32)
    slot_of = np.zeros(cap, dtype=np.int32)
    brick_of = np.zeros(cap, dtype=np.int32)
    voxel_of = np.zeros(cap, dtype=np.int32)
    n_steps = np.zeros(R, dtype=np.int32)
    amb = np.zeros(R, dtype=np.int32)
    n = lib().or_active_samples(C.byref(g), C.byref(r), C.byref(s), brick, _ptr(ray_of), _ptr(slot_of),
                                _ptr(brick_of), _ptr(voxel_of), cap, _ptr(n_steps), _ptr(amb))
    if n < 0:
        raise ValueError("capacity too small")
    return {"ray": ray_of[:n], "slot": slot_of[:n], "brick": brick_of[:n], "voxel": voxel_of[:n],
            "n_steps": n_steps, "amb": amb.astype(bool)}


def sample_grid(grid, points):
    keep = _Keep()
    g = _grid(grid, keep)
    p = np.ascontiguousarray(points, dtype=np.float64)
    n = p.shape[0]
    raw = np.zeros(n)
    feat = np.zeros((n, grid.C))
    lib().or_sample_grid(C.byref(g), _ptr(p), n, _ptr(raw), _ptr(feat))
    return raw, feat


def mlp_eval(mlp, x):
    keep = _Keep()
    m = _mlp(mlp, keep)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], 3))
    lib().or_mlp_eval(C.byref(m), _ptr(x), x.shape[0], _ptr(out))
    return out


def encode(mlp, feat, d):
    keep = _Keep()
    m = _mlp(mlp, keep)
    feat = np.ascontiguousarray(feat, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    M, Cn = feat.shape
    x = np.zeros((M, mlp.in_dim))
    lib().or_encode(C.byref(m), Cn, _ptr(feat), _ptr(d), M, _ptr(x))
    return x


def warp(ref_rgb, ref_depth, ref_cam, tgt_cam, max_angle_deg: float = 180.0, void_grid=None,
         void_sampling=None) -> dict:
    """SpaRW warp of a float32 reference frame into the target camera (FP32 decisions)."""
    keep = _Keep()
    rgb = keep(np.ascontiguousarray(ref_rgb, dtype=np.float32))
    dep = keep(np.ascontiguousarray(ref_depth, dtype=np.float32))
    rc, tc = _cam(ref_cam), _cam(tgt_cam)
    NT = tgt_cam.width * tgt_cam.height
    out = {"rgb": np.zeros((NT, 3), dtype=np.float32), "depth": np.zeros(NT, dtype=np.float32),
           "mask": np.zeros(NT, dtype=np.uint8), "hole_idx": np.zeros(NT, dtype=np.int32),
           "src": np.zeros(NT, dtype=np.int32)}
    nh = C.c_int32(0)
    vg = _grid(void_grid, keep) if void_grid is not None else None
    vs = _sampling(void_sampling or tgt_cam.sampling)
    r = lib().or_warp(_ptr(rgb), _ptr(dep), C.byref(rc), C.byref(tc), max_angle_deg,
                      C.byref(vg) if vg is not None else None, C.byref(vs), _ptr(out["rgb"]),
                      _ptr(out["depth"]), _ptr(out["mask"]), _ptr(out["hole_idx"]), C.byref(nh), _ptr(out["src"]))
    if r != 0:
        raise MemoryError("or_warp")
    out["n_holes"] = int(nh.value)
    out["hole_idx"] = out["hole_idx"][: out["n_holes"]]
    return out


def warp_bruteforce(ref_depth, ref_cam, tgt_cam, max_angle_deg: float = 180.0):
    dep = np.ascontiguousarray(ref_depth, dtype=np.float32)
    rc, tc = _cam(ref_cam), _cam(tgt_cam)
    src = np.zeros(tgt_cam.width * tgt_cam.height, dtype=np.int32)
    lib().or_warp_bruteforce(_ptr(dep), C.byref(rc), C.byref(tc), max_angle_deg, _ptr(src))
    return src


def rel_pose(ref_cam, tgt_cam):
    rc, tc = _cam(ref_cam), _cam(tgt_cam)
    out = np.zeros(12, dtype=np.float32)
    lib().or_rel_pose(C.byref(rc), C.byref(tc), _ptr(out))
    return out.reshape(3, 4)


def backward(grid, mlp, sampling, d_rgb, cam=None, pix=None, rays=None, with_mlp: bool = False):
    """FP64 gradient of a loss with dL/drgb = ``d_rgb`` w.r.t. density, features (and MLP)."""
    keep = _Keep()
    g, m, s = _grid(grid, keep), _mlp(mlp, keep), _sampling(sampling)
    r = _rays(keep, cam, pix, rays)
    dr = np.ascontiguousarray(d_rgb, dtype=np.float64)
    dd = np.zeros(grid.density.size)
    df = np.zeros(grid.features.size)
    nm = mlp.flat().size
    dm = np.zeros(nm) if with_mlp else None
    rc = lib().or_backward(C.byref(g), C.byref(m), C.byref(r), C.byref(s), _ptr(dr), _ptr(dd), _ptr(df), _ptr(dm))
    if rc != 0:
        raise ValueError(f"or_backward failed ({rc})")
    return dd.reshape(grid.density.shape), df.reshape(grid.features.shape), dm


def relu_margin(grid, mlp, sampling, cam=None, pix=None, rays=None):
    keep = _Keep()
    g, m, s = _grid(grid, keep), _mlp(mlp, keep), _sampling(sampling)
    r = _rays(keep, cam, pix, rays)
    out = np.zeros(_nrays(cam, pix, rays))
    lib().or_relu_margin(C.byref(g), C.byref(m), C.byref(r), C.byref(s), _ptr(out))
    return out


def extrapolate_pose(c2w_prev, c2w_cur, lead: float) -> np.ndarray:
    """Pose of a reference frame extrapolated from the two latest camera poses (Sec. III-C, Eq. 5-6),
    in FP64.  c2w are 3x4 [R | position] camera-to-world matrices one frame interval apart.

    Eq. 5: v = (T_cur - T_prev) / dt.  Eq. 6: T_ref = T_cur + v t_r with t_r = lead * dt (the paper
    takes lead = N / 2).  The paper writes the velocity of the position only; the orientation is
    extrapolated the same way with the angular velocity: the rotation dR = R_cur R_prev^T taken from
    prev to cur is applied `lead` more times (its axis-angle form, angle scaled by lead):
    R_ref = rot(axis, lead * angle) R_cur."""
    P = np.asarray(c2w_prev, dtype=np.float64).reshape(3, 4)
    Cm = np.asarray(c2w_cur, dtype=np.float64).reshape(3, 4)
    pos = Cm[:, 3] + lead * (Cm[:, 3] - P[:, 3])
    dR = Cm[:, :3] @ P[:, :3].T
    angle = math.acos(min(1.0, max(-1.0, (np.trace(dR) - 1.0) / 2.0)))
    if angle < 1e-12:
        Rl = np.eye(3)
    else:
        axis = np.array([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]]) / (2.0 * math.sin(angle))
        a = lead * angle
        K = np.array([[0.0, -axis[2], axis[1]], [axis[2], 0.0, -axis[0]], [-axis[1], axis[0], 0.0]])
        Rl = np.eye(3) + math.sin(a) * K + (1.0 - math.cos(a)) * (K @ K)  # Rodrigues
    return np.concatenate([Rl @ Cm[:, :3], pos[:, None]], axis=1)


def reference_schedule(n_frames: int, window: int, lead: str = "centred"):
    """Which poses each reference frame of a trajectory is extrapolated from (Sec. III-C,
    Eq. 5-6), for the overlapped pipeline: frames come in windows of ``window`` targets and window
    w is warped from reference w.  Reference 0 is frame 0 itself (``None``).  Reference w >= 1 is
    rendered while window w - 1 runs, so it uses the two latest poses known when window w - 1
    starts: frames s - 1 and s with s the first frame of window w - 1 (at least 1, since two poses
    are needed).  Its lead, in frame intervals after frame s: "centred" carries it to the centre of
    the window it serves, frame w * window + window / 2; "paper" is Eq. 6 read literally,
    t_r = N / 2 with N = window.  Returns one (prev, cur, lead) triple per window."""
    out = [None]
    for w in range(1, (n_frames + window - 1) // window):
        s = max(1, (w - 1) * window)
        centre = w * window + window / 2.0
        out.append((s - 1, s, centre - s if lead == "centred" else window / 2.0))
    return out


def upsample_bilinear(img, W: int, H: int) -> np.ndarray:
    """Bilinear resampling of img [h, w, C] to [H, W, C] in FP64 (the DS-2 comparator: the frame is
    rendered at half resolution, then upsampled by bilinear interpolation).  Reading: pixel
    centres align, so output pixel (i, j) samples the source at ((i + 1/2) w / W - 1/2,
    (j + 1/2) h / H - 1/2); coordinates are clamped to the image."""
    img = np.asarray(img, dtype=np.float64)
    h, w = img.shape[:2]
    u = np.clip((np.arange(W) + 0.5) * w / W - 0.5, 0.0, w - 1)
    v = np.clip((np.arange(H) + 0.5) * h / H - 0.5, 0.0, h - 1)
    x0, y0 = np.floor(u).astype(int), np.floor(v).astype(int)
    x1, y1 = np.minimum(x0 + 1, w - 1), np.minimum(y0 + 1, h - 1)
    fx, fy = (u - x0)[None, :, None], (v - y0)[:, None, None]
    top = img[y0][:, x0] * (1 - fx) + img[y0][:, x1] * fx
    bot = img[y1][:, x0] * (1 - fx) + img[y1][:, x1] * fx
    return top * (1 - fy) + bot * fy


def hash_features(grid, points):
    """Hash-encoding features of a grid with ``hash`` at world points [n, 3] -> [n, levels * feat]."""
    keep = _Keep()
    g = _grid(grid, keep)
    p = keep(np.ascontiguousarray(points, dtype=np.float64))
    out = np.zeros((p.shape[0], grid.C))
    lib().or_hash_features(C.byref(g), _ptr(p), p.shape[0], _ptr(out))
    return out


def camera_rays(cam, pix=None) -> dict:
    """The oracle's rays of camera ``cam`` (every pixel, or the list ``pix``): FP32 origin and
    direction (``o32``, ``d32``, the rays of the integer decisions) and FP64 (``o64``, ``d64``)."""
    keep = _Keep()
    r = _rays(keep, cam=cam, pix=pix)
    n = _nrays(cam=cam, pix=pix)
    out = {"o32": np.zeros((n, 3), np.float32), "d32": np.zeros((n, 3), np.float32),
           "o64": np.zeros((n, 3)), "d64": np.zeros((n, 3))}
    lib().or_rays_of(C.byref(r), _ptr(out["o32"]), _ptr(out["d32"]), _ptr(out["o64"]), _ptr(out["d64"]))
    return out


def max_threads() -> int:
    return int(lib().or_max_threads())


def psnr(a, b) -> float:
    mse = float(np.mean((np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
