"""Seeded synthetic inputs for the voxel-grid NeRF + SpaRW hot path.

This module only draws numbers and lays them out in memory: density and
feature grids, occupancy masks, MLP weights, camera poses and explicit rays.
It holds none of the rendering or warping arithmetic; the oracle (``oracle/``)
and the CUDA library (``paper_2404_11852_gb300``) both consume exactly the
arrays produced here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``
and a uniform double is ``(z >> 11) * 2**-53``.  Every array is therefore
identical on every machine and numpy version.

The scenes stand in for the paper's Synthetic-NeRF scenes (Sec. V, "Datasets"),
which are not available: DirectVoxGO-like dense grids of density and features
(Sec. II-B) built from Gaussian blobs and smoothed noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# fixed seeds of the standard workloads
SEED_SCENE = 1234
SEED_MLP = 5678
SEED_RAYS = 91011


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> int:
    """A sub-stream seed derived from (seed, tag) by one SplitMix64 step."""
    z = np.array([(seed * 1_000_003 + tag * 7919 + 1) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return int(_mix(z)[0])


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the stream ``seed`` as uint64."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
    return _mix(z)


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """``n`` float64 draws, uniform on [lo, hi)."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


# --------------------------------------------------------------------------------------------
# containers


@dataclass
class HashGrid:
    """Multiresolution hash encoding: ``table`` is [levels][2^log2_size][feat]; level l divides the
    box into ``res[l]`` cells per axis."""

    levels: int
    feat: int
    log2_size: int
    res: tuple
    table: np.ndarray


@dataclass
class Grid:
    """Dense voxel grid: ``density`` is [Nz][Ny][Nx], ``features`` is [Nz][Ny][Nx][C].

    Vertices sit on the corners of the axis-aligned box ``aabb_min .. aabb_max``.
    ``occ`` is an optional [R][R][R] uint8 occupancy mask over the same box.  With ``hash`` set,
    the colour features come from that encoding (C = levels * feat) and ``features`` is unused.
    """

    n: tuple
    C: int
    density: np.ndarray
    features: np.ndarray
    aabb_min: tuple = (-1.0, -1.0, -1.0)
    aabb_max: tuple = (1.0, 1.0, 1.0)
    act_shift: float = -4.0
    occ: np.ndarray | None = None
    hash: HashGrid | None = None

    @property
    def occ_res(self) -> int:
        return 0 if self.occ is None else int(self.occ.shape[0])

    def astype(self, dtype) -> "Grid":
        return Grid(self.n, self.C, self.density.astype(dtype), self.features.astype(dtype),
                    self.aabb_min, self.aabb_max, self.act_shift, self.occ, self.hash)


@dataclass
class Mlp:
    """Weights of the view-dependent colour MLP, row-major [out][in], float32."""

    w1: np.ndarray
    b1: np.ndarray
    w2: np.ndarray
    b2: np.ndarray
    w3: np.ndarray
    b3: np.ndarray
    n_freq: int = 4

    @property
    def in_dim(self) -> int:
        return int(self.w1.shape[1])

    @property
    def hidden(self) -> int:
        return int(self.w1.shape[0])

    def flat(self) -> np.ndarray:
        return np.concatenate([a.ravel() for a in (self.w1, self.b1, self.w2, self.b2, self.w3, self.b3)])


@dataclass
class Sampling:
    """How slots are placed along a ray and when the march stops.

    ``step == 0``: ``n_samples`` midpoints between ``near`` and ``far``.
    ``step > 0``: slots every ``step`` from the ray's entry into the box, at most
    ``n_samples`` of them and only while inside the box.
    """

    near: float = 0.5
    far: float = 2.5
    n_samples: int = 64
    step: float = 0.0
    t_stop: float = 1e-3
    bg: tuple = (0.0, 0.0, 0.0)
    void_acc: float = 0.5


@dataclass
class Camera:
    """Pinhole camera; ``c2w`` is row-major 3x4 with OpenCV axes (x right, y down, z forward)."""

    width: int
    height: int
    f: float
    cx: float
    cy: float
    c2w: np.ndarray  # float32 [3, 4]
    sampling: Sampling = field(default_factory=Sampling)


# --------------------------------------------------------------------------------------------
# grids


def blob_density(N: int, n_blobs: int, seed: int, aabb=(-1.0, 1.0), amp_scale: float = 1.0) -> np.ndarray:
    """Sum of isotropic Gaussian blobs sampled at the vertices, float64 [N][N][N].

    Per blob, in draw order: centre (x, y, z) ~ U[-0.6, 0.6], width s ~ U[0.06, 0.2],
    amplitude A ~ amp_scale U[10, 40]; the value at vertex p is A * exp(-|p - mu|^2 / (2 s^2)).
    """
    d = uniform(stream_seed(seed, 1), 5 * n_blobs)
    lo, hi = aabb
    x = lo + (hi - lo) * np.arange(N, dtype=np.float64) / (N - 1)
    raw = np.zeros((N, N, N), dtype=np.float64)
    for b in range(n_blobs):
        mu = -0.6 + 1.2 * d[5 * b: 5 * b + 3]
        s = 0.06 + 0.14 * d[5 * b + 3]
        amp = amp_scale * (10.0 + 30.0 * d[5 * b + 4])
        gx = np.exp(-((x - mu[0]) ** 2) / (2 * s * s))
        gy = np.exp(-((x - mu[1]) ** 2) / (2 * s * s))
        gz = np.exp(-((x - mu[2]) ** 2) / (2 * s * s))
        raw += amp * (gz[:, None, None] * (gy[None, :, None] * gx[None, None, :]))
    return raw


def smoothed_features(N: int, C: int, seed: int) -> np.ndarray:
    """Uniform [-1, 1] noise in memory order [z][y][x][c], then one [1,2,1]/4 pass
    along x, y and z with the edge vertex repeated.  float32 [N][N][N][C]."""
    s = stream_seed(seed, 2)
    out = np.empty((N, N, N, C), dtype=np.float32)
    plane = N * N * C
    for z in range(N):
        out[z] = uniform(s, plane, -1.0, 1.0, offset=z * plane).astype(np.float32).reshape(N, N, C)
    q = np.float32(0.25)
    for axis in (2, 1, 0):
        a = np.moveaxis(out, axis, 0)
        sm = np.empty_like(a)
        sm[1:-1] = (a[:-2] + 2.0 * a[1:-1] + a[2:]) * q
        sm[0] = (a[0] + 2.0 * a[0] + a[1]) * q
        sm[-1] = (a[-2] + 2.0 * a[-1] + a[-1]) * q
        out = np.ascontiguousarray(np.moveaxis(sm, 0, axis))
    return out


def occupancy_mask(raw: np.ndarray, R: int, frac: float) -> np.ndarray:
    """[R][R][R] uint8 mask marking the ceil(frac * R^3) cells whose largest vertex value
    (over the vertices inside or on the cell) is largest; ties go to the lower cell index."""
    N = raw.shape[0]
    lo = [-(-k * (N - 1) // R) for k in range(R)]
    hi = [((k + 1) * (N - 1)) // R for k in range(R)]

    def reduce(a, axis):
        parts = [np.take(a, np.arange(lo[k], hi[k] + 1), axis=axis).max(axis=axis, keepdims=True)
                 for k in range(R)]
        return np.concatenate(parts, axis=axis)

    m = reduce(reduce(reduce(raw, 2), 1), 0)
    k = int(math.ceil(frac * R ** 3))
    order = np.argsort(-m.ravel(), kind="stable")[:k]
    occ = np.zeros(R ** 3, dtype=np.uint8)
    occ[order] = 1
    return occ.reshape(R, R, R)


def make_grid(N: int, C: int, n_blobs: int, seed: int = SEED_SCENE, dtype=np.float32,
              occ_res: int = 0, occ_frac: float = 0.15, amp_scale: float = 1.0) -> Grid:
    raw = blob_density(N, n_blobs, seed, amp_scale=amp_scale)
    feat = smoothed_features(N, C, seed)
    occ = occupancy_mask(raw, occ_res, occ_frac) if occ_res else None
    return Grid((N, N, N), C, raw.astype(dtype), feat.astype(dtype), occ=occ)


def affine_grid(N: int, C: int, a: np.ndarray, b: np.ndarray, dtype=np.float64,
                aabb=(-1.0, 1.0)) -> Grid:
    """Grid whose channel values are exactly a[c] + b[c] . p at every vertex p
    (channel 0 of ``a``/``b`` goes to the density, 1.. to the features)."""
    lo, hi = aabb
    x = lo + (hi - lo) * np.arange(N, dtype=np.float64) / (N - 1)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    chans = [a[c] + b[c, 0] * X + b[c, 1] * Y + b[c, 2] * Z for c in range(C + 1)]
    dens = chans[0].astype(dtype)
    feat = np.stack(chans[1:], axis=-1).astype(dtype)
    return Grid((N, N, N), C, dens, feat, (lo,) * 3, (hi,) * 3)


# --------------------------------------------------------------------------------------------
# MLP


def make_mlp(C: int, seed: int = SEED_MLP, hidden: int = 128, n_freq: int = 4,
             random_bias: bool = False) -> Mlp:
    """Xavier-uniform weights (+-sqrt(6 / (fan_in + fan_out))); biases zero unless
    ``random_bias`` (then U[-0.5, 0.5])."""
    in_dim = C + 3 + 6 * n_freq
    shapes = [(hidden, in_dim), (hidden, hidden), (3, hidden)]
    ws, bs = [], []
    for i, (o, k) in enumerate(shapes):
        a = math.sqrt(6.0 / (o + k))
        ws.append(uniform(stream_seed(seed, 10 + i), o * k, -a, a).astype(np.float32).reshape(o, k))
        if random_bias:
            bs.append(uniform(stream_seed(seed, 20 + i), o, -0.5, 0.5).astype(np.float32))
        else:
            bs.append(np.zeros(o, dtype=np.float32))
    return Mlp(ws[0], bs[0], ws[1], bs[1], ws[2], bs[2], n_freq)


# --------------------------------------------------------------------------------------------
# cameras and rays


def look_at_c2w(eye: np.ndarray, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world 3x4 (float64) with OpenCV axes: z toward ``target``, y down."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, dtype=np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.concatenate([np.stack([x, y, z], axis=1), eye[:, None]], axis=1)


def orbit_camera(width: int, height: int, fov_deg: float = 40.0, radius: float = 1.5,
                 az_deg: float = 30.0, el_deg: float = 20.0,
                 sampling: Sampling | None = None) -> Camera:
    az, el = math.radians(az_deg), math.radians(el_deg)
    eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return Camera(width, height, float(np.float32(f)), width / 2.0, height / 2.0,
                  look_at_c2w(eye).astype(np.float32), sampling or Sampling())


def _rodrigues(axis: np.ndarray, ang: float) -> np.ndarray:
    a = axis / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def offset_camera(ref: Camera, k: int, yaw_deg: float = 1.0, shift: float = 0.005) -> Camera:
    """Target pose ``k`` steps from ``ref``: k * yaw_deg about the camera's own up axis
    (-y_c) and k * shift along its x axis (head-motion-like trajectory)."""
    c2w = ref.c2w.astype(np.float64)
    R, t = c2w[:, :3], c2w[:, 3]
    rot = _rodrigues(-R[:, 1], math.radians(k * yaw_deg))
    R2 = rot @ R
    t2 = t + k * shift * R[:, 0]
    out = np.concatenate([R2, t2[:, None]], axis=1).astype(np.float32)
    return Camera(ref.width, ref.height, ref.f, ref.cx, ref.cy, out, ref.sampling)


SPARW_OFFSETS = tuple(list(range(-8, 0)) + list(range(1, 9)))


def random_rays(R: int, seed: int = SEED_RAYS, radius: float = 1.5, aim: float = 0.5):
    """Origins uniform on the sphere of ``radius``, each aimed at a point ~ U[-aim, aim]^3.
    Returns float32 (o [R,3], d [R,3]) with |d| = 1 to float32 rounding."""
    u = uniform(stream_seed(seed, 30), 5 * R).reshape(R, 5)
    zc = 2.0 * u[:, 0] - 1.0
    ph = 2.0 * math.pi * u[:, 1]
    rr = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    o = radius * np.stack([rr * np.cos(ph), rr * np.sin(ph), zc], axis=1)
    p = -aim + 2.0 * aim * u[:, 2:5]
    d = p - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def random_targets(R: int, seed: int = SEED_RAYS) -> np.ndarray:
    return uniform(stream_seed(seed, 31), 3 * R).reshape(R, 3).astype(np.float32)


# --------------------------------------------------------------------------------------------
# the standard workloads


def hash_levels(levels: int, base_res: int, max_res: int) -> tuple:
    """Cells per axis of each level: floor(base * b^l) with b = (max / base)^(1 / (levels - 1))."""
    b = math.exp((math.log(max_res) - math.log(base_res)) / max(levels - 1, 1))
    return tuple(int(math.floor(base_res * b ** l)) for l in range(levels))


def make_hash_grid(levels: int = 8, feat: int = 2, log2_size: int = 19, base_res: int = 16, max_res: int = 512,
                   seed: int = SEED_SCENE, dtype=np.float16) -> HashGrid:
    """Table entries U[-1, 1] (a seeded stand-in for trained features)."""
    T = 1 << log2_size
    table = uniform(stream_seed(seed, 40), levels * T * feat, -1.0, 1.0).astype(dtype).reshape(levels, T, feat)
    return HashGrid(levels, feat, log2_size, hash_levels(levels, base_res, max_res), table)


def with_hash(g: Grid, h: HashGrid) -> Grid:
    """The scene g (density, occupancy, box) with its colour features from the hash encoding h."""
    return Grid(g.n, h.levels * h.feat, g.density, None, g.aabb_min, g.aabb_max, g.act_shift, g.occ, h)


def scene_small(dtype=np.float32) -> Grid:
    """64^3 grid, 8 blobs, 12 feature channels (the small single-view scene)."""
    return make_grid(64, 12, 8, SEED_SCENE, dtype)


OPAQUE_AMP_SCALE = 25.0


def scene_small_opaque(dtype=np.float32) -> Grid:
    """The small scene with every blob amplitude x 25 (A ~ U[250, 1000]): a ray stops within a
    sample or two of entering a blob, so the expected depth is the blob's surface, as with the
    solid objects of the paper's scenes (the fog-like default blobs composite ~100 samples)."""
    return make_grid(64, 12, 8, SEED_SCENE, dtype, amp_scale=OPAQUE_AMP_SCALE)


def scene_large() -> Grid:
    """256^3 grid, 24 blobs, FP16 density and features (416 MB), 32^3 mask at 15 %."""
    return make_grid(256, 12, 24, SEED_SCENE, np.float16, occ_res=32, occ_frac=0.15)


def scene_backward() -> Grid:
    """160^3 x 12 FP32 grid with 8 blobs (the training-step scene)."""
    return make_grid(160, 12, 8, SEED_SCENE, np.float32)


def scene_fd() -> Grid:
    """16^3 x 4 grid for finite-difference checks."""
    return make_grid(16, 4, 8, SEED_SCENE, np.float64)


def sampling_uniform(n_samples: int = 64, t_stop: float = 1e-3) -> Sampling:
    return Sampling(near=0.5, far=2.5, n_samples=n_samples, step=0.0, t_stop=t_stop)


def sampling_march(N: int = 256, max_samples: int = 256) -> Sampling:
    """Slots every half voxel from the box entry, at most ``max_samples``."""
    h = 2.0 / (N - 1)
    return Sampling(near=0.0, far=1e30, n_samples=max_samples, step=float(np.float32(0.5 * h)),
                    t_stop=1e-3)
