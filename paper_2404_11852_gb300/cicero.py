"""Python binding of libcicero (include/cicero.h): argument marshalling only.

Every function named ``cicero_*`` here calls the C entry point of the same name with the raw
device pointers of the torch tensors it is given and raises ``CiceroError`` when the status is
not ``CICERO_OK``.  All computation happens in the CUDA kernels of the library; if the library
is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcicero.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_ALIGNMENT, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_INTERNAL = range(8)
F32, F16 = 0, 1
MLP_FP32, MLP_BF16, MLP_FP32_SPLIT = 0, 1, 2


class CiceroError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cicero status {status}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("C", C.c_int), ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3),
                ("act_shift", C.c_float), ("dtype", C.c_int), ("density", C.c_void_p), ("features", C.c_void_p),
                ("occ", C.c_void_p), ("occ_res", C.c_int)]


class Mlp(C.Structure):
    _fields_ = [("in_dim", C.c_int), ("hidden", C.c_int), ("n_freq", C.c_int), ("w1", C.c_void_p),
                ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p), ("w3", C.c_void_p), ("b3", C.c_void_p)]


class Sampling(C.Structure):
    _fields_ = [("near_t", C.c_float), ("far_t", C.c_float), ("n_samples", C.c_int), ("step", C.c_float),
                ("t_stop", C.c_float), ("bg", C.c_float * 3), ("void_acc", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("f", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("c2w", C.c_float * 12)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("brick", C.c_int), ("max_records", C.c_longlong), ("mlp_groups", C.c_int)]


class HashGridDesc(C.Structure):
    _fields_ = [("levels", C.c_int), ("features", C.c_int), ("log2_size", C.c_int), ("res", C.c_int * 16),
                ("dtype", C.c_int), ("table", C.c_void_p)]


class Job(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("mlp", C.c_void_p), ("cam", C.c_void_p), ("sampling", C.c_void_p),
                ("rgb", C.c_void_p), ("depth", C.c_void_p)]


_P = C.c_void_p
_Z = C.c_size_t
_SIGS = {
    "cicero_render": ([_P] * 10 + [_Z, _P], C.c_int),
    "cicero_render_rays": ([_P] * 4 + [C.c_int] + [_P] * 7 + [_Z, _P], C.c_int),
    "cicero_render_holes": ([_P] * 7 + [C.c_int] + [_P] * 3 + [_Z, _P], C.c_int),
    "cicero_render_workspace_size": ([_P, C.c_int, _P, _P], _Z),
    "cicero_render_holes_batch": ([_P, _P, _P, C.c_int, _P, _P, _P, _P, C.c_int, _P, _P, _P, _Z, _P], C.c_int),
    "cicero_warp": ([_P] * 4 + [C.c_float] + [_P] * 8 + [_Z, _P], C.c_int),
    "cicero_warp_workspace_size": ([_P], _Z),
    "cicero_warp_batch": ([_P] * 3 + [_P, C.c_int, C.c_float] + [_P] * 7 + [_P, _Z, _P], C.c_int),
    "cicero_warp_batch_workspace_size": ([_P, C.c_int], _Z),
    "cicero_warp_noalloc": ([_P] * 4 + [C.c_float] + [_P] * 8, C.c_int),
    "cicero_render_backward": ([_P] * 4 + [C.c_int] + [_P] * 6 + [_Z, _P], C.c_int),
    "cicero_backward_workspace_size": ([_P, C.c_int, _P], _Z),
    "cicero_backward_mlp_workspace_size": ([_P, C.c_int, _P], _Z),
    "cicero_build_rit": ([_P] * 8 + [_Z, _P], C.c_int),
    "cicero_build_rit_workspace_size": ([_P] * 4, _Z),
    "cicero_mlp_eval": ([_P, _P, C.c_int, C.c_int, _P, _P, _Z, _P], C.c_int),
    "cicero_mlp_eval_workspace_size": ([C.c_int], _Z),
    "cicero_workspace_status": ([_P, _P], C.c_int),
    "cicero_autotune_brick": ([_P] * 4 + [C.c_int] + [_P] * 3 + [_Z] + [_P] * 3, C.c_int),
    "cicero_batch_workspace_size": ([_P, C.c_int, _P], _Z),
    "cicero_batch_table_bytes": ([C.c_int], _Z),
    "cicero_batch_create": ([_P, C.c_int, _P, _P, _Z, _P], C.c_int),
    "cicero_batch_launch": ([_P, _P], C.c_int),
    "cicero_batch_destroy": ([_P], C.c_int),
    "cicero_batch_autotune": ([_P, C.c_int, _P, _P, _Z, _P, _P, _P], C.c_int),
    "cicero_extrapolate_pose": ([_P, _P, C.c_float, _P], C.c_int),
    "cicero_render_hash": ([_P] * 8 + [_P, _Z, _P], C.c_int),
    "cicero_render_hash_workspace_size": ([_P, _P, C.c_int, _P, _P], _Z),
    "cicero_upsample_bilinear": ([_P, C.c_int, C.c_int, C.c_int, _P, C.c_int, C.c_int, _P], C.c_int),
    "cicero_pipeline_workspace_size": ([_P, _P, _P, _P, C.c_int, C.c_longlong], _Z),
    "cicero_pipeline_create": ([_P] * 5 + [C.c_int, C.c_longlong, C.c_float, _P, _Z, _P], C.c_int),
    "cicero_pipeline_run": ([_P, _P, C.c_int, C.c_int, _P, _P, _P, _P], C.c_int),
    "cicero_reference_poses": ([_P, C.c_int, C.c_int, C.c_int, _P], C.c_int),
    "cicero_pipeline_status": ([_P, _P], C.c_int),
    "cicero_pipeline_destroy": ([_P], C.c_int),
    "cicero_profile_begin": ([], C.c_int),
    "cicero_profile_end": ([_P, _P, C.c_int], C.c_int),
    "cicero_launch_count": ([], C.c_longlong),
    "cicero_last_error": ([], C.c_char_p),
    "cicero_version": ([], C.c_char_p),
}

_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcicero.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise CiceroError(status, lib().cicero_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ws(ws: torch.Tensor):
    return _ptr(ws), C.c_size_t(ws.numel() * ws.element_size())


def _ref(x):
    return None if x is None else C.byref(x)


# ---------------------------------------------------------------------------------------------
# descriptors


class DeviceGrid:
    """A grid resident on the GPU: torch tensors plus the ``cicero_grid`` descriptor."""

    def __init__(self, density: torch.Tensor, features: torch.Tensor | None, aabb_min=(-1.0, -1.0, -1.0),
                 aabb_max=(1.0, 1.0, 1.0), act_shift: float = -4.0, occ: torch.Tensor | None = None):
        """features may be None for a grid whose colour features come from a hash encoding."""
        assert features is None or density.dtype == features.dtype
        assert density.dtype in (torch.float32, torch.float16)
        self.density, self.occ = density.contiguous(), occ
        self.features = features.contiguous() if features is not None else None
        nz, ny, nx = density.shape
        d = Grid()
        d.n[:] = [nx, ny, nz]
        d.C = features.shape[3] if features is not None else 0
        d.aabb_min[:] = list(aabb_min)
        d.aabb_max[:] = list(aabb_max)
        d.act_shift = act_shift
        d.dtype = F16 if density.dtype == torch.float16 else F32
        d.density = self.density.data_ptr()
        d.features = self.features.data_ptr() if self.features is not None else None
        if occ is not None:
            self.occ = occ.to(torch.uint8).contiguous()
            d.occ = self.occ.data_ptr()
            d.occ_res = self.occ.shape[0]
        self.desc = d

    @classmethod
    def from_host(cls, g, device="cuda"):
        """From a host grid object with numpy ``density``/``features``/``occ`` arrays."""
        dens = torch.from_numpy(g.density).to(device)
        feat = torch.from_numpy(g.features).to(device) if g.features is not None else None
        occ = None if g.occ is None else torch.from_numpy(g.occ).to(device)
        return cls(dens, feat, g.aabb_min, g.aabb_max, g.act_shift, occ)


class DeviceMlp:
    def __init__(self, w1, b1, w2, b2, w3, b3, n_freq: int = 4):
        self.t = [w.contiguous().float() for w in (w1, b1, w2, b2, w3, b3)]
        m = Mlp()
        m.hidden, m.in_dim = self.t[0].shape
        m.n_freq = n_freq
        m.w1, m.b1, m.w2, m.b2, m.w3, m.b3 = [w.data_ptr() for w in self.t]
        self.desc = m

    @classmethod
    def from_host(cls, m, device="cuda"):
        return cls(*[torch.from_numpy(a).to(device) for a in (m.w1, m.b1, m.w2, m.b2, m.w3, m.b3)], n_freq=m.n_freq)


def sampling(near=0.5, far=2.5, n_samples=64, step=0.0, t_stop=1e-3, bg=(0.0, 0.0, 0.0), void_acc=0.5) -> Sampling:
    s = Sampling()
    s.near_t, s.far_t, s.n_samples, s.step, s.t_stop = near, far, n_samples, step, t_stop
    s.bg[:] = list(bg)
    s.void_acc = void_acc
    return s


def sampling_from(sp) -> Sampling:
    return sampling(sp.near, sp.far, sp.n_samples, sp.step, sp.t_stop, sp.bg, sp.void_acc)


def camera(width, height, f, cx, cy, c2w) -> Camera:
    c = Camera()
    c.width, c.height, c.f, c.cx, c.cy = width, height, f, cx, cy
    c.c2w[:] = [float(v) for v in c2w.reshape(-1)]
    return c


def camera_from(cam) -> Camera:
    return camera(cam.width, cam.height, cam.f, cam.cx, cam.cy, cam.c2w)


def options(precision: int = MLP_FP32, brick: int = 8, max_records: int = 0, mlp_groups: int = 0) -> Options:
    o = Options()
    o.precision, o.brick, o.max_records, o.mlp_groups = precision, brick, max_records, mlp_groups
    return o


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)


def cicero_render(grid: Grid, mlp: Mlp, cam: Camera, samp: Sampling, opt: Options | None, rgb, depth, acc, n_steps,
                  ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_render(C.byref(grid), C.byref(mlp), C.byref(cam), C.byref(samp), _ref(opt), _ptr(rgb),
                               _ptr(depth), _ptr(acc), _ptr(n_steps), p, n, _stream(stream)))


def cicero_render_rays(grid: Grid, mlp: Mlp, ray_o, ray_d, samp: Sampling, opt: Options | None, rgb, depth, acc,
                       n_steps, ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_render_rays(C.byref(grid), C.byref(mlp), _ptr(ray_o), _ptr(ray_d), ray_o.shape[0],
                                    C.byref(samp), _ref(opt), _ptr(rgb), _ptr(depth), _ptr(acc), _ptr(n_steps), p, n,
                                    _stream(stream)))


def cicero_render_holes(grid: Grid, mlp: Mlp, cam: Camera, samp: Sampling, opt: Options | None, hole_idx, n_holes,
                        max_holes: int, rgb_inout, depth_inout, ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_render_holes(C.byref(grid), C.byref(mlp), C.byref(cam), C.byref(samp), _ref(opt),
                                     _ptr(hole_idx), _ptr(n_holes), int(max_holes), _ptr(rgb_inout),
                                     _ptr(depth_inout), p, n, _stream(stream)))


def cicero_render_holes_batch(grid: Grid, mlp: Mlp, cams, samp: Sampling, opt: Options | None, hole_idx, n_holes,
                              max_rays: int, rgb_inout, depth_inout, ws, stream=None):
    """cams: list of Camera; hole_idx / rgb_inout / depth_inout: lists of CUDA tensors (depth may be
    None); n_holes: one int32 CUDA tensor holding the per-view counts contiguously."""
    V = len(cams)
    cam_arr = (Camera * V)(*cams)
    P = C.c_void_p * V
    h = P(*[t.data_ptr() for t in hole_idx])
    rgb = P(*[t.data_ptr() for t in rgb_inout])
    dep = P(*[(t.data_ptr() if t is not None else None) for t in depth_inout]) if depth_inout is not None else None
    assert n_holes.is_cuda and n_holes.is_contiguous() and n_holes.numel() == V
    p, n = _ws(ws)
    _check(lib().cicero_render_holes_batch(C.byref(grid), C.byref(mlp), cam_arr, V, C.byref(samp), _ref(opt), h,
                                           _ptr(n_holes), int(max_rays), rgb, dep, p, n, _stream(stream)))


def cicero_render_workspace_size(grid: Grid, n_rays: int, samp: Sampling, opt: Options | None = None) -> int:
    return int(lib().cicero_render_workspace_size(C.byref(grid), int(n_rays), C.byref(samp), _ref(opt)))


def cicero_warp(ref_rgb, ref_depth, ref_cam: Camera, tgt_cam: Camera, max_angle_deg: float, void_grid: Grid | None,
                void_samp: Sampling | None, warped_rgb, warped_depth, hole_mask, hole_idx, n_holes, ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_warp(_ptr(ref_rgb), _ptr(ref_depth), C.byref(ref_cam), C.byref(tgt_cam), float(max_angle_deg),
                             _ref(void_grid), _ref(void_samp), _ptr(warped_rgb), _ptr(warped_depth), _ptr(hole_mask),
                             _ptr(hole_idx), _ptr(n_holes), p, n, _stream(stream)))


def cicero_warp_noalloc(ref_rgb, ref_depth, ref_cam: Camera, tgt_cam: Camera, max_angle_deg: float,
                        void_grid: Grid | None, void_samp: Sampling | None, warped_rgb, warped_depth, hole_mask,
                        hole_idx, n_holes, stream=None):
    _check(lib().cicero_warp_noalloc(_ptr(ref_rgb), _ptr(ref_depth), C.byref(ref_cam), C.byref(tgt_cam),
                                     float(max_angle_deg), _ref(void_grid), _ref(void_samp), _ptr(warped_rgb),
                                     _ptr(warped_depth), _ptr(hole_mask), _ptr(hole_idx), _ptr(n_holes),
                                     _stream(stream)))


def cicero_warp_batch(ref_rgb, ref_depth, ref_cam: Camera, tgt_cams, max_angle_deg: float, void_grid: Grid | None,
                      void_samp: Sampling | None, warped_rgb, warped_depth, hole_mask, hole_idx, n_holes, ws,
                      stream=None):
    """tgt_cams: list of Camera; warped_* / hole_*: lists of CUDA tensors (warped_depth may be None);
    n_holes: one int32 CUDA tensor with len(tgt_cams) entries."""
    V = len(tgt_cams)
    P = C.c_void_p * V
    arr = lambda ts: P(*[(t.data_ptr() if t is not None else None) for t in ts])
    p, n = _ws(ws)
    assert n_holes.is_cuda and n_holes.is_contiguous() and n_holes.numel() == V
    _check(lib().cicero_warp_batch(_ptr(ref_rgb), _ptr(ref_depth), C.byref(ref_cam), (Camera * V)(*tgt_cams), V,
                                   float(max_angle_deg), _ref(void_grid), _ref(void_samp), arr(warped_rgb),
                                   arr(warped_depth) if warped_depth is not None else None, arr(hole_mask),
                                   arr(hole_idx), _ptr(n_holes), p, n, _stream(stream)))


def cicero_warp_batch_workspace_size(tgt_cams) -> int:
    V = len(tgt_cams)
    return int(lib().cicero_warp_batch_workspace_size((Camera * V)(*tgt_cams), V))


def cicero_warp_workspace_size(tgt_cam: Camera) -> int:
    return int(lib().cicero_warp_workspace_size(C.byref(tgt_cam)))


def cicero_render_backward(grid: Grid, mlp: Mlp, ray_o, ray_d, samp: Sampling, d_rgb, d_density, d_features, d_mlp,
                           ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_render_backward(C.byref(grid), C.byref(mlp), _ptr(ray_o), _ptr(ray_d), ray_o.shape[0],
                                        C.byref(samp), _ptr(d_rgb), _ptr(d_density), _ptr(d_features), _ptr(d_mlp),
                                        p, n, _stream(stream)))


def cicero_backward_workspace_size(grid: Grid, n_rays: int, samp: Sampling) -> int:
    return int(lib().cicero_backward_workspace_size(C.byref(grid), int(n_rays), C.byref(samp)))


def cicero_backward_mlp_workspace_size(grid: Grid, n_rays: int, samp: Sampling) -> int:
    return int(lib().cicero_backward_mlp_workspace_size(C.byref(grid), int(n_rays), C.byref(samp)))


def cicero_build_rit(grid: Grid, cam: Camera, samp: Sampling, opt: Options | None, brick_offsets, samples, ws,
                     stream=None) -> int:
    p, n = _ws(ws)
    nb = C.c_int(0)
    _check(lib().cicero_build_rit(C.byref(grid), C.byref(cam), C.byref(samp), _ref(opt), _ptr(brick_offsets),
                                  _ptr(samples), C.byref(nb), p, n, _stream(stream)))
    return int(nb.value)


def cicero_autotune_brick(grid: Grid, mlp: Mlp, cam: Camera, samp: Sampling, precision: int, rgb, depth, ws,
                          stream=None):
    """Returns (best brick, {brick: ms})."""
    p, n = _ws(ws)
    best = C.c_int(0)
    ms = (C.c_float * 3)()
    _check(lib().cicero_autotune_brick(C.byref(grid), C.byref(mlp), C.byref(cam), C.byref(samp), int(precision),
                                       _ptr(rgb), _ptr(depth), p, n, _stream(stream), C.byref(best), ms))
    return int(best.value), {b: float(ms[i]) for i, b in enumerate((4, 8, 16))}


def cicero_build_rit_workspace_size(grid: Grid, cam: Camera, samp: Sampling, opt: Options | None = None) -> int:
    return int(lib().cicero_build_rit_workspace_size(C.byref(grid), C.byref(cam), C.byref(samp), _ref(opt)))


def cicero_mlp_eval(mlp: Mlp, x, precision: int, c, ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_mlp_eval(C.byref(mlp), _ptr(x), x.shape[0], int(precision), _ptr(c), p, n, _stream(stream)))


def cicero_mlp_eval_workspace_size(M: int) -> int:
    return int(lib().cicero_mlp_eval_workspace_size(int(M)))


def cicero_workspace_status(ws, stream=None):
    _check(lib().cicero_workspace_status(_ptr(ws), _stream(stream)))


STAGES = ("march", "bucket", "gather_mlp", "composite", "warp_splat", "warp_resolve", "bwd_ray", "bwd_brick",
          "mlp_eval", "bwd_weights")


def cicero_profile_begin():
    _check(lib().cicero_profile_begin())


def cicero_profile_end() -> dict:
    n = len(STAGES)
    ms = (C.c_double * n)()
    cnt = (C.c_longlong * n)()
    _check(lib().cicero_profile_end(ms, cnt, n))
    return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}


def cicero_launch_count() -> int:
    return int(lib().cicero_launch_count())


def cicero_version() -> str:
    return lib().cicero_version().decode()


# ---------------------------------------------------------------------------------------------
# batched rendering


def jobs_array(jobs) -> C.Array:
    """A ``cicero_job`` array from (grid desc, mlp desc, camera, sampling, rgb tensor, depth tensor or
    None) tuples; the descriptor structs must stay referenced while the array is used."""
    arr = (Job * len(jobs))()
    for i, (g, m, cam, samp, rgb, depth) in enumerate(jobs):
        arr[i].grid = C.addressof(g)
        arr[i].mlp = C.addressof(m)
        arr[i].cam = C.addressof(cam)
        arr[i].sampling = C.addressof(samp)
        arr[i].rgb = _ptr(rgb).value
        arr[i].depth = _ptr(depth).value if depth is not None else None
    return arr


def cicero_batch_workspace_size(jobs, opt: Options) -> int:
    return int(lib().cicero_batch_workspace_size(jobs, len(jobs), C.byref(opt)))


def cicero_batch_table_bytes(n_jobs: int) -> int:
    return int(lib().cicero_batch_table_bytes(int(n_jobs)))


class Batch:
    """A planned batch (``cicero_batch`` handle); ``launch`` renders every job again."""

    def __init__(self, jobs, opt: Options, ws: torch.Tensor):
        p, n = _ws(ws)
        h = C.c_void_p()
        _check(lib().cicero_batch_create(jobs, len(jobs), C.byref(opt), p, n, C.byref(h)))
        self.handle, self.ws, self.n_jobs = h, ws, len(jobs)

    def launch(self, stream=None):
        _check(lib().cicero_batch_launch(self.handle, _stream(stream)))

    def status(self, stream=None):
        """Raise if a kernel of the last launches reported an error."""
        off = cicero_batch_table_bytes(self.n_jobs)
        _check(lib().cicero_workspace_status(C.c_void_p(self.ws.data_ptr() + off), _stream(stream)))

    def header(self):
        off = cicero_batch_table_bytes(self.n_jobs)
        return self.ws[off:off + 64].view(torch.int32).cpu()

    def close(self):
        if self.handle:
            lib().cicero_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cicero_batch_autotune(jobs, opt: Options, ws: torch.Tensor, stream=None):
    """Returns the fastest Options (brick and mlp_groups set) and the timed ms per (brick, mlp_groups)."""
    p, n = _ws(ws)
    best = Options()
    ms = (C.c_float * 12)()
    _check(lib().cicero_batch_autotune(jobs, len(jobs), C.byref(opt), p, n, _stream(stream), C.byref(best), ms))
    return best, {(b, g): float(ms[4 * i + g - 1]) for i, b in enumerate((4, 8, 16)) for g in range(1, 5)}


def cicero_extrapolate_pose(prev: Camera, cur: Camera, lead: float) -> Camera:
    out = Camera()
    _check(lib().cicero_extrapolate_pose(C.byref(prev), C.byref(cur), float(lead), C.byref(out)))
    return out


# ---------------------------------------------------------------------------------------------
# SpaRW over a trajectory


def cicero_pipeline_workspace_size(grid: Grid, cam: Camera, samp: Sampling, opt: Options, window: int,
                                   hole_records: int) -> int:
    return int(lib().cicero_pipeline_workspace_size(C.byref(grid), C.byref(cam), C.byref(samp), C.byref(opt),
                                                    int(window), int(hole_records)))


class Pipeline:
    """A ``cicero_pipeline`` handle: SpaRW windows with the next reference rendered on a second stream."""

    def __init__(self, grid: Grid, mlp: Mlp, cam: Camera, samp: Sampling, opt: Options, window: int,
                 hole_records: int, max_angle_deg: float, ws: torch.Tensor):
        p, n = _ws(ws)
        h = C.c_void_p()
        _check(lib().cicero_pipeline_create(C.byref(grid), C.byref(mlp), C.byref(cam), C.byref(samp), C.byref(opt),
                                            int(window), int(hole_records), float(max_angle_deg), p, n, C.byref(h)))
        self.handle, self.ws, self.window = h, ws, window

    def run(self, targets, rgb, depth=None, lead: str = "centred", stream_tgt=None, stream_ref=None):
        """targets: list of Camera; rgb / depth: lists of device tensors (one per target)."""
        tg = (Camera * len(targets))(*targets)
        pr = (C.c_void_p * len(rgb))(*[_ptr(t).value for t in rgb])
        pd = (C.c_void_p * len(depth))(*[_ptr(t).value for t in depth]) if depth is not None else None
        _check(lib().cicero_pipeline_run(self.handle, tg, len(targets), _LEADS[lead], pr, pd, _stream(stream_tgt),
                                         _stream(stream_ref)))

    def status(self, stream=None):
        _check(lib().cicero_pipeline_status(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            lib().cicero_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


LEAD_CENTRED, LEAD_PAPER = 0, 1
_LEADS = {"centred": LEAD_CENTRED, "paper": LEAD_PAPER}


def cicero_reference_poses(targets, window: int, lead: str = "centred"):
    """Reference cameras the pipeline derives from a trajectory (list of Camera); lead is
    "centred" or "paper"."""
    tg = (Camera * len(targets))(*targets)
    n_win = (len(targets) + window - 1) // window
    out = (Camera * n_win)()
    _check(lib().cicero_reference_poses(tg, len(targets), int(window), _LEADS[lead], out))
    return list(out)


def cicero_upsample_bilinear(src, w: int, h: int, dst, W: int, H: int, stream=None):
    """src [h*w][C] -> dst [H*W][C] (device FP32 tensors)."""
    ch = src.numel() // (w * h)
    _check(lib().cicero_upsample_bilinear(_ptr(src), int(w), int(h), int(ch), _ptr(dst), int(W), int(H),
                                          _stream(stream)))


# ---------------------------------------------------------------------------------------------
# hash-encoded rendering


class DeviceHashGrid:
    """A hash encoding resident on the GPU (scenes.HashGrid -> torch tensor + descriptor)."""

    def __init__(self, table: torch.Tensor, res, log2_size: int):
        assert table.dtype in (torch.float16, torch.float32) and table.shape[-1] == 2
        self.table = table.contiguous()
        d = HashGridDesc()
        d.levels, d.features, d.log2_size = table.shape[0], 2, int(log2_size)
        d.res[: len(res)] = list(res)
        d.dtype = F16 if table.dtype == torch.float16 else F32
        d.table = self.table.data_ptr()
        self.desc = d

    @classmethod
    def from_host(cls, h, device="cuda"):
        return cls(torch.from_numpy(h.table).to(device), h.res, h.log2_size)


def cicero_render_hash(grid: Grid, hg: HashGridDesc, mlp: Mlp, cam: Camera, samp: Sampling, opt: Options, rgb, depth,
                       ws, stream=None):
    p, n = _ws(ws)
    _check(lib().cicero_render_hash(C.byref(grid), C.byref(hg), C.byref(mlp), C.byref(cam), C.byref(samp),
                                    C.byref(opt), _ptr(rgb), _ptr(depth), p, n, _stream(stream)))


def cicero_render_hash_workspace_size(grid: Grid, hg: HashGridDesc, n_rays: int, samp: Sampling, opt: Options) -> int:
    return int(lib().cicero_render_hash_workspace_size(C.byref(grid), C.byref(hg), int(n_rays), C.byref(samp),
                                                       C.byref(opt)))
