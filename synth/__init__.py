"""Seeded synthetic inputs shared by the CUDA library's tests/benchmarks and the oracle.

This package only makes inputs (textures, grids, query coordinates, footprints); it
holds none of the filtering arithmetic.  The heavy loops are plain C
(``noise.c``), built on first use with the host C compiler.  Workload shapes:

* 2D: RGBA float32 value-noise texture (4 octaves, gain 1/2, values in [0, 1]) and
  uniform texture coordinates.
* dense 3D: fractal-noise density thresholded at a percentile (70th: ~30% of voxels
  non-zero), values (n - thr) / (1 - thr).
* sparse 3D: a cloud-like field on the 8^3-leaf cell grid (fBm times a radial
  falloff), thresholded so that a target fraction of leaves is active (threshold
  calibrated on a seeded subsample), fine fBm voxel values inside active leaves.
* ray-march queries: a pinhole camera on a sphere around the grid centre looking at
  the centre, a fixed number of jittered samples per ray.
* material: a 7-channel texture (RGB albedo, unit normal xyz, roughness).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "noise.c")
_LIB_PATH = os.path.join(_HERE, "_noise.so")
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)


def build(force=False):
    """Compile noise.c into a shared library next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32, i32, i64, dbl = ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_fbm2_image.argtypes = [u32, i32, i32, i32, dbl, i32, dbl, _f32p]
        lib.synth_fbm3_grid.argtypes = [u32, i32, i32, i32, i64, i64, i64, dbl, i32, dbl, _f32p]
        lib.synth_cloud_cells.argtypes = [u32, i32, dbl, i32, dbl, dbl, _f32p]
        lib.synth_leaf_values.argtypes = [u32, i64, ctypes.POINTER(ctypes.c_int32), dbl, i32, dbl, _f32p]
        lib.synth_camera_queries.argtypes = [u32, i32, i32, i32, dp, dbl, dp, dbl, dbl, _f32p]
        lib.synth_uniform.argtypes = [u32, u32, i64, _f32p]
        for f in (lib.synth_fbm2_image, lib.synth_fbm3_grid, lib.synth_cloud_cells,
                  lib.synth_leaf_values, lib.synth_camera_queries, lib.synth_uniform):
            f.restype = None
        _lib = lib
    return _lib


def _fp(a):
    return a.ctypes.data_as(_f32p)


def uniform(n, seed, stream=0):
    """n float32 values, uniform in [0, 1)."""
    out = np.empty(int(n), dtype=np.float32)
    _L().synth_uniform(seed, stream, int(n), _fp(out))
    return out


def texture2d(W=256, H=256, C=4, seed=1, octaves=4, gain=0.5, period=None):
    """Value-noise image, float32 (H, W, C), each channel normalised to [0, 1]."""
    out = np.empty((H, W, C), dtype=np.float32)
    period = float(period if period is not None else max(W, H) / 8.0)
    _L().synth_fbm2_image(seed, W, H, C, period, octaves, gain, _fp(out))
    return out


def uv_queries(n, seed=2):
    """n texture coordinates, uniform in [0, 1)^2, float32 (n, 2)."""
    return np.stack([uniform(n, seed, 0), uniform(n, seed, 1)], axis=1)


def lods(n, seed, lo=0.0, hi=4.0):
    """n level-of-detail values (log2 footprints), uniform in [lo, hi)."""
    return (np.float32(lo) + uniform(n, seed, 7) * np.float32(hi - lo)).astype(np.float32)


def dense_density(n=256, seed=3, keep_frac=0.30, octaves=5, gain=0.5, period=48.0):
    """Fractal-noise density, float32 (n, n, n) indexed [z, y, x]; the top keep_frac
    of voxels are non-zero with values (v - thr) / (1 - thr)."""
    g = np.empty((n, n, n), dtype=np.float32)
    _L().synth_fbm3_grid(seed, n, n, n, 0, 0, 0, period, octaves, gain, _fp(g))
    thr = np.float32(np.quantile(g.reshape(-1)[:: max(1, g.size // (1 << 22))], 1.0 - keep_frac))
    return (np.maximum(g - thr, 0) / (np.float32(1) - thr)).astype(np.float32)


def sparse_cloud(domain=2048, seed=4, active_frac=0.04, cell_octaves=4, voxel_octaves=5,
                 gain=0.5):
    """Cloud-like sparse grid over [0, domain)^3 with 8^3 leaves.

    Returns (origins int32 (L, 3) multiples of 8, values float32 (L, 512) laid out
    [x][y][z] within each leaf)."""
    n = domain // 8
    cells = np.empty((n, n, n), dtype=np.float32)          # [z, y, x]
    _L().synth_cloud_cells(seed, n, n / 6.0, cell_octaves, gain, 0.5, _fp(cells))
    rng = np.random.default_rng(seed)
    sample = cells.reshape(-1)[rng.integers(0, cells.size, size=min(cells.size, 1 << 20))]
    thr = np.quantile(sample, 1.0 - active_frac)
    z, y, x = np.nonzero(cells > thr)
    origins = (np.stack([x, y, z], axis=1) * 8).astype(np.int32)
    values = np.empty((origins.shape[0], 512), dtype=np.float32)
    if origins.shape[0]:
        oc = np.ascontiguousarray(origins)
        _L().synth_leaf_values(seed + 17, oc.shape[0],
                               oc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 24.0,
                               voxel_octaves, gain, _fp(values))
    return origins, values


def camera_queries(W, H, steps, centre, radius, half_span, seed, fov_deg=40.0):
    """Ray-march sample positions, float32 (W*H*steps, 3), ray-major / step-minor.
    The camera direction is a seeded random unit vector."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    v = np.ascontiguousarray(v / np.linalg.norm(v), dtype=np.float64)
    c = np.ascontiguousarray(np.asarray(centre, dtype=np.float64))
    out = np.empty((W * H * steps, 3), dtype=np.float32)
    dp = ctypes.POINTER(ctypes.c_double)
    _L().synth_camera_queries(seed, W, H, steps, c.ctypes.data_as(dp), float(radius),
                              v.ctypes.data_as(dp), float(fov_deg), float(half_span), _fp(out))
    return out


def material(size=4096, seed=5):
    """7-channel material texture float32 (size, size, 7): RGB albedo in [0, 1], a unit
    normal (xyz) from the slopes of a height field, roughness in [0.05, 1]."""
    rgb = texture2d(size, size, 3, seed=seed, octaves=5, period=size / 16.0)
    h = texture2d(size, size, 1, seed=seed + 1, octaves=6, period=size / 32.0)[..., 0]
    rough = texture2d(size, size, 1, seed=seed + 2, octaves=4, period=size / 8.0)[..., 0]
    gx = (np.roll(h, -1, axis=1) - np.roll(h, 1, axis=1)) * np.float32(8.0)
    gy = (np.roll(h, -1, axis=0) - np.roll(h, 1, axis=0)) * np.float32(8.0)
    inv = np.float32(1) / np.sqrt(gx * gx + gy * gy + np.float32(1))
    out = np.empty((size, size, 7), dtype=np.float32)
    out[..., 0:3] = rgb
    out[..., 3] = -gx * inv
    out[..., 4] = -gy * inv
    out[..., 5] = inv
    out[..., 6] = np.float32(0.05) + np.float32(0.95) * rough
    return out


# Full-size workload recipes (the shapes of the paper's workloads, synthetic data).
C2_RAYS = dict(W=1920, H=1080, steps=16, centre=(128.0, 128.0, 128.0), radius=384.0,
               half_span=222.0, seed=3)
C3_RAYS = dict(W=2048, H=2048, steps=16, centre=(1024.0, 1024.0, 1024.0), radius=3072.0,
               half_span=1774.0, seed=4)


def box_levels(level0, num_levels):
    """Box-filtered pyramid of a power-of-two image (H, W, C): level L texel = mean of
    the level-0 block it covers.  Returns a list of float32 arrays."""
    base = np.asarray(level0, dtype=np.float64)
    H, W, C = base.shape
    out = [np.asarray(level0, dtype=np.float32)]
    for L in range(1, num_levels):
        hl, wl = max(1, H >> L), max(1, W >> L)
        out.append(base.reshape(hl, H // hl, wl, W // wl, C).mean(axis=(1, 3)).astype(np.float32))
    return out


def neural_init(size, latent_levels, seed=5, latent_scale=0.5):
    """Initial neural-texture state: latents ~ N(0, latent_scale^2) for every texel of
    the latent levels ([level][y][x][8] concatenated) and He-initialised decoder
    weights with zero biases, flat (W1 8x64, b1, W2 64x64, b2, W3 64x7, b3)."""
    rng = np.random.default_rng(seed)
    n = sum(max(1, size >> L) ** 2 for L in range(latent_levels))
    latents = (rng.standard_normal((n, 8)) * latent_scale).astype(np.float32)
    parts = []
    for fan_in, shape in ((8, (8, 64)), (64, (64,)), (64, (64, 64)), (64, (64,)), (64, (64, 7)), (7, (7,))):
        if len(shape) == 2:
            parts.append(rng.standard_normal(shape).reshape(-1) * np.sqrt(2.0 / shape[0]))
        else:
            parts.append(np.zeros(shape[0]))
    return latents, np.concatenate(parts).astype(np.float32)


def plane_view(W=1920, H=1080, seed=7, fov_deg=60.0, height=0.04, pitch_deg=12.0):
    """Texture coordinates and their screen-space derivatives for a camera looking
    across a textured ground plane (the textured square [0, 1]^2 of z = 0, uv = (x, y)),
    the grazing view where footprints are long ellipses (Section 5.2's anisotropic
    test scene is a textured plane).  The camera stands at a seeded point near the
    y = 0 edge, `height` above the plane, yawed by a seeded angle, pitched down by
    `pitch_deg`.  Per pixel whose ray hits the square: uv of the hit point and
    (du/dx, dv/dx, du/dy, dv/dy), the differences to the hits of the rays through the
    neighbouring pixels (+1 in x, +1 in y).  Returns (uv (n, 2), grad (n, 4)) float32."""
    rng = np.random.default_rng(seed)
    eye = np.array([rng.uniform(0.35, 0.65), rng.uniform(-0.05, 0.05), height])
    yaw = np.radians(rng.uniform(-20.0, 20.0))
    pitch = np.radians(-pitch_deg)
    fwd = np.array([np.sin(yaw) * np.cos(pitch), np.cos(yaw) * np.cos(pitch), np.sin(pitch)])
    right = np.array([np.cos(yaw), -np.sin(yaw), 0.0])
    up = np.cross(right, fwd)
    t = np.tan(np.radians(fov_deg) / 2)

    def hits(px, py):
        sx = (2 * (px + 0.5) / W - 1) * t * W / H
        sy = (1 - 2 * (py + 0.5) / H) * t
        d = fwd[None] + sx[:, None] * right[None] + sy[:, None] * up[None]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = -eye[2] / d[:, 2]
        p = eye[None] + s[:, None] * d
        return p[:, :2], s

    py, px = np.mgrid[0:H, 0:W]
    px, py = px.ravel().astype(np.float64), py.ravel().astype(np.float64)
    p, s = hits(px, py)
    px1, s1 = hits(px + 1, py)
    py1, s2 = hits(px, py + 1)
    ok = (s > 0) & (s1 > 0) & (s2 > 0) & np.all((p >= 0) & (p < 1), axis=1)
    uv = p[ok]
    grad = np.concatenate([px1[ok] - uv, py1[ok] - uv], axis=1)
    return uv.astype(np.float32), grad.astype(np.float32)


def sphere_points(n, seed=8, centre=(0.5, 0.5, 0.5), radius=0.45):
    """Surface points of a sphere with their unit normals (triplanar-mapping queries):
    directions uniform on the sphere (normalised Gaussian vectors).  Returns
    (positions (n, 3), normals (n, 3)) float32."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = np.asarray(centre)[None] + radius * d
    return p.astype(np.float32), d.astype(np.float32)
