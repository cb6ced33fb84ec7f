"""Seeded synthetic inputs for the Katsevich reconstruction tests and benchmark.

This module is the input generator shared by the FP64 oracle tests and the GPU
path's tests and benchmark.  It holds the workload descriptions (the primary
scan/volume parameters of each configuration), seeded ellipsoid phantoms,
their exact FP64 line integrals through a helical scan with a curved detector,
and seeded Gaussian noise.  It holds none of the reconstruction method's
arithmetic: derived geometry (fan angle, detector spacing, pitch) is computed
by each side from the primary parameters below.

Geometry dictionaries passed to :func:`project` use these keys (plain numbers):
``R, D, P, lambda0, z0, lambda_first, views_per_turn, n_views, n_rows, n_cols,
d_alpha, alpha_offset, d_w, w_offset, nx, ny, nz, dx, dy, dz, x0, y0, z_first``.

Phantom recipe (no published phantom table is reproduced here):

* ``shepp_style``: a nested head-like set built by a fixed rule -- an outer
  ellipsoid of density 1, an interior ellipsoid of density -0.8 (net 0.2), and
  6-8 small inner ellipsoids with seeded centres, semi-axes and densities.
* ``random_ellipsoids``: U{20..40} ellipsoids, centres uniform in the disc of
  radius 0.5 x (volume half-width) and uniform over the volume's z extent,
  semi-axes U[10, 120] mm, uniformly random rotations, densities U[0.1, 1].
* ``ball``: a single uniform ball (used for accuracy pins).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")

# ---------------------------------------------------------------------------
# Workloads: primary parameters only.
# ---------------------------------------------------------------------------
CONFIGS = {
    1: dict(name="fp32_det32x128_vol64x64x32", R=500.0, D=1000.0, views_per_turn=128, turns=3,
            n_rows=32, n_cols=128, n_cols_full=128, col_keep=1, det_half_width=32.0,
            nx=64, ny=64, nz=32, voxel=1.0, pitch_factor=1.0,
            phantom="shepp_style", noise_sigma=1e-3, batch=1, seed=1),
    2: dict(name="fp32_det64x736_vol512x512x256", R=595.0, D=1085.6, views_per_turn=1160, turns=8,
            n_rows=64, n_cols=736, n_cols_full=736, col_keep=1, det_half_width=256.0,
            nx=512, ny=512, nz=256, voxel=1.0, pitch_factor=1.0,
            phantom="random_ellipsoids", noise_sigma=0.0, batch=1, seed=2),
    3: dict(name="diff_det64x368_vol256x256x64_b4", R=595.0, D=1085.6, views_per_turn=580, turns=4,
            n_rows=64, n_cols=368, n_cols_full=736, col_keep=2, det_half_width=256.0,
            nx=256, ny=256, nz=64, voxel=1.0, pitch_factor=1.5,
            phantom="random_ellipsoids", noise_sigma=0.0, batch=4, seed=3),
    4: dict(name="mixed_det64x736_vol512x512x256", R=595.0, D=1085.6, views_per_turn=1160, turns=8,
            n_rows=64, n_cols=736, n_cols_full=736, col_keep=1, det_half_width=256.0,
            nx=512, ny=512, nz=256, voxel=1.0, pitch_factor=1.0,
            phantom="random_ellipsoids", noise_sigma=0.0, batch=1, seed=4),
}


def config(index: int) -> dict:
    """A copy of workload ``index``'s primary parameters."""
    return dict(CONFIGS[index])


def phantom_seed(index: int) -> int:
    return 1000 + index


def noise_seed(index: int) -> int:
    return 2000 + index


# ---------------------------------------------------------------------------
# Native line-integral library
# ---------------------------------------------------------------------------
class _Scan(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("D", ctypes.c_double), ("P", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("z0", ctypes.c_double),
                ("lambda_first", ctypes.c_double), ("dlam", ctypes.c_double),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("d_alpha", ctypes.c_double), ("alpha_offset", ctypes.c_double),
                ("d_w", ctypes.c_double), ("w_offset", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the FP64 projector (gcc, OpenMP) into synth/_build/libsynth.so."""
    src = os.path.join(_HERE, "project.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-D_GNU_SOURCE", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_project.argtypes = [ctypes.POINTER(_Scan), dp, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, dp]
        lib.synth_project_rays.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
        lib.synth_density.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, dp, dp]
        lib.synth_ray.argtypes = [ctypes.POINTER(_Scan), ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp, dp]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _scan(geom: dict) -> _Scan:
    return _Scan(R=geom["R"], D=geom["D"], P=geom["P"], lambda0=geom["lambda0"], z0=geom["z0"],
                 lambda_first=geom["lambda_first"], dlam=2.0 * math.pi / geom["views_per_turn"],
                 n_rows=geom["n_rows"], n_cols=geom["n_cols"], d_alpha=geom["d_alpha"],
                 alpha_offset=geom["alpha_offset"], d_w=geom["d_w"], w_offset=geom["w_offset"])


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------
def _rotation(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of the unit quaternion q = (w, x, y, z)."""
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipsoid(center, axes, rho, rotation=None) -> np.ndarray:
    """One 14-double ellipsoid record: centre, quadric matrix, density, bound."""
    Q = np.eye(3) if rotation is None else np.asarray(rotation, dtype=np.float64)
    a = np.asarray(axes, dtype=np.float64)
    M = Q @ np.diag(1.0 / (a * a)) @ Q.T
    rec = np.empty(14)
    rec[0:3] = center
    rec[3:12] = M.reshape(-1)
    rec[12] = rho
    rec[13] = float(a.max()) * (1.0 + 1e-12)
    return rec


def ball(center, radius, rho=1.0) -> np.ndarray:
    return ellipsoid(center, (radius, radius, radius), rho)[None, :]


def shepp_style(seed: int, half_width: float, z_center: float) -> np.ndarray:
    """Nested head-like ellipsoid set built by a fixed, seeded rule."""
    rng = np.random.default_rng(seed)
    r0 = 0.9 * half_width
    recs = [ellipsoid((0.0, 0.0, z_center), (0.80 * r0, 0.70 * r0, 1.5 * r0), 1.0),
            ellipsoid((0.0, 0.0, z_center), (0.74 * r0, 0.64 * r0, 1.4 * r0), -0.8)]
    n_inner = int(rng.integers(6, 9))
    for _ in range(n_inner):
        ax = rng.uniform(0.08, 0.25, size=3) * r0
        lim = 0.55 * r0 - ax.max()
        cx, cy = rng.uniform(-lim, lim, size=2) * np.array([0.74 / 0.8, 0.64 / 0.8])
        cz = z_center + rng.uniform(-0.8, 0.8) * r0
        q = rng.normal(size=4)
        recs.append(ellipsoid((cx, cy, cz), ax, float(rng.uniform(-0.1, 0.3)), _rotation(q)))
    return np.stack(recs)


def random_ellipsoids(seed: int, half_width: float, z_lo: float, z_hi: float) -> np.ndarray:
    """U{20..40} random ellipsoids inside the volume's central disc."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 41))
    recs = []
    for _ in range(n):
        rad = 0.5 * half_width * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        c = (rad * math.cos(th), rad * math.sin(th), rng.uniform(z_lo, z_hi))
        ax = rng.uniform(10.0, 120.0, size=3)
        q = rng.normal(size=4)
        recs.append(ellipsoid(c, ax, float(rng.uniform(0.1, 1.0)), _rotation(q)))
    return np.stack(recs)


def phantom_for(cfg: dict, geom: dict, seed: int) -> np.ndarray:
    """The phantom named by a workload, placed in the geometry's volume."""
    half = 0.5 * min(geom["nx"] * geom["dx"], geom["ny"] * geom["dy"])
    zc = geom["z_first"] + 0.5 * (geom["nz"] - 1) * geom["dz"]
    if cfg["phantom"] == "shepp_style":
        return shepp_style(seed, half, zc)
    if cfg["phantom"] == "random_ellipsoids":
        zh = 0.5 * geom["nz"] * geom["dz"]
        return random_ellipsoids(seed, half, zc - zh, zc + zh)
    if cfg["phantom"] == "ball":
        return ball((0.0, 0.0, zc), 0.6 * half)
    raise ValueError(cfg["phantom"])


# ---------------------------------------------------------------------------
# Projection and noise
# ---------------------------------------------------------------------------
def project(geom: dict, ellipsoids: np.ndarray, v_begin: int = 0, n_views: int | None = None) -> np.ndarray:
    """FP64 line integrals g[view][row][col] of the phantom for the helical scan."""
    lib = _load()
    if n_views is None:
        n_views = geom["n_views"] - v_begin
    e = np.ascontiguousarray(ellipsoids, dtype=np.float64)
    out = np.empty((n_views, geom["n_rows"], geom["n_cols"]), dtype=np.float64)
    sc = _scan(geom)
    lib.synth_project(ctypes.byref(sc), _dp(e), e.shape[0], v_begin, n_views, _dp(out))
    return out


def project_rays(ellipsoids: np.ndarray, src: np.ndarray, direction: np.ndarray) -> np.ndarray:
    lib = _load()
    e = np.ascontiguousarray(ellipsoids, dtype=np.float64)
    s = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(direction, dtype=np.float64).reshape(-1, 3)
    out = np.empty(s.shape[0])
    lib.synth_project_rays(_dp(e), e.shape[0], s.shape[0], _dp(s), _dp(d), _dp(out))
    return out


def ray(geom: dict, lam: float, alpha: float, w: float):
    """Source point and unit direction of the ray (lam, alpha, w)."""
    lib = _load()
    s = np.empty(3)
    d = np.empty(3)
    sc = _scan(geom)
    lib.synth_ray(ctypes.byref(sc), lam, alpha, w, _dp(s), _dp(d))
    return s, d


def density(ellipsoids: np.ndarray, points: np.ndarray) -> np.ndarray:
    lib = _load()
    e = np.ascontiguousarray(ellipsoids, dtype=np.float64)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty(p.shape[0])
    lib.synth_density(_dp(e), e.shape[0], p.shape[0], _dp(p), _dp(out))
    return out


def add_noise(sino: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Additive seeded Gaussian noise N(0, sigma^2)."""
    if sigma <= 0:
        return sino
    rng = np.random.default_rng(seed)
    return sino + rng.normal(0.0, sigma, size=sino.shape)


def random_sino(shape, seed: int) -> np.ndarray:
    """Seeded standard-normal array (for linearity/adjoint tests)."""
    return np.random.default_rng(seed).normal(size=shape)
