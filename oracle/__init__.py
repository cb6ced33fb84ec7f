"""FP64 CPU oracle of the Katsevich helical cone-beam reconstruction operator.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library (``paper_2201_02309_b300``) and never imports it.

The arithmetic lives in ``katsevich_oracle.c`` (the reconstruction operator)
and ``simulate_oracle.c`` (data simulation: helical projection, sparse
detector upsampling, Gaussian+Poisson noise), plain C, FP64, OpenMP; this
module only compiles them, marshals numpy arrays, and derives a workload's
geometry from its primary parameters (its own copy of those rules).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "katsevich_oracle.c")
_SRC_SIM = os.path.join(_HERE, "simulate_oracle.c")
_HDR = os.path.join(_HERE, "katsevich_oracle.h")

GEOM_KEYS = ["R", "D", "P", "lambda0", "z0", "lambda_first", "views_per_turn", "n_views",
             "n_rows", "n_cols", "d_alpha", "alpha_offset", "d_w", "w_offset",
             "nx", "ny", "nz", "dx", "dy", "dz", "x0", "y0", "z_first", "n_psi", "endpoint_mode"]


class _Geom(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("D", ctypes.c_double), ("P", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("z0", ctypes.c_double), ("lambda_first", ctypes.c_double),
                ("views_per_turn", ctypes.c_int64), ("n_views", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("d_alpha", ctypes.c_double), ("alpha_offset", ctypes.c_double),
                ("d_w", ctypes.c_double), ("w_offset", ctypes.c_double),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z_first", ctypes.c_double),
                ("n_psi", ctypes.c_int64), ("endpoint_mode", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, OpenMP, no fast-math) into oracle/_build/liboracle.so."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_SIM), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                           "-fno-fast-math", "-ffp-contract=off", _SRC, _SRC_SIM, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None
_D = ctypes.c_double
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PG = ctypes.POINTER(_Geom)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "or_r_fov": (_D, [_PG]),
        "or_alpha_m": (_D, [_PG]),
        "or_fit_pitch": (_D, [_D, _D, _I64, _D, _D]),
        "or_w_kappa": (_D, [_PG, _D, _D]),
        "or_w_td_top": (_D, [_PG, _D]),
        "or_w_td_bottom": (_D, [_PG, _D]),
        "or_psi_hat": (ctypes.c_int, [_PG, _D, _D, _PD]),
        "or_pi_endpoints": (None, [_PG, _D, _D, _D, _PD, _PD]),
        "or_project_point": (None, [_PG, _D, _D, _D, _D, _PD, _PD, _PD]),
        "or_kappa_table": (None, [_PG, _PI32, _PD]),
        "or_psi_table": (None, [_PG, _PI32, _PD]),
        "or_pi_table": (None, [_PG, _PI32, _PI32, _PD, _PD, _PD, _PD]),
        "or_derivative": (None, [_PG, _PD, _I64, _PD]),
        "or_length_weight": (None, [_PG, _PD, _I64]),
        "or_forward_rebin": (None, [_PG, _PI32, _PD, _PD, _I64, _PD]),
        "or_hilbert": (None, [_PG, _PD, _I64, _PD]),
        "or_backward_rebin": (None, [_PG, _PI32, _PD, _PD, _I64, _PD]),
        "or_post_cosine": (None, [_PG, _PD, _I64]),
        "or_filter": (None, [_PG, _PI32, _PD, _PI32, _PD, _PD, _I64, _PD]),
        "or_backproject": (ctypes.c_int, [_PG, _PI32, _PI32, _PD, _PD, _PD, _I64, _I64, _PD]),
        "or_pi_window_points": (None, [_PG, _I64, _PI64, _PI64, _PI64, _PD, _PD]),
        "or_backproject_points": (ctypes.c_int, [_PG, _PD, _I64, _I64, _I64, _PI64, _PI64, _PI64,
                                                 _PD, _PD, _PD]),
        "or_backproject_adjoint": (ctypes.c_int, [_PG, _PI32, _PI32, _PD, _PD, _PD, _PD, _I64, _I64]),
        "or_filter_adjoint": (None, [_PG, _PI32, _PD, _PI32, _PD, _PD, _I64, _PD]),
        "or_extents": (None, [_PG, _PI32, _PI32, _PD, _PD, _PD]),
        "or_update_count": (_I64, [_PG, _PI32, _PI32]),
        "or_ray": (None, [_PG, _I64, _I64, _I64, _PD, _PD]),
        "or_project": (None, [_PG, _PD, _I64, _I64, _PD]),
        "or_sparse_upsample": (None, [_PG, _PD, _I64, _I64, _PD]),
        "or_philox4x32_10": (None, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                    ctypes.POINTER(ctypes.c_uint32)]),
        "or_poisson": (_I64, [_D, ctypes.c_uint64, _I64]),
        "or_gaussian": (_D, [ctypes.c_uint64, _I64]),
        "or_add_noise": (None, [_PD, _I64, _D, _D, _D, ctypes.c_uint64, _PD, _PI64, _PD]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    if a.dtype == np.float64:
        return a.ctypes.data_as(_PD)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_PI32)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_PI64)
    raise TypeError(a.dtype)


def _g(geom: dict) -> _Geom:
    return _Geom(**{k: geom[k] for k in GEOM_KEYS})


# ---------------------------------------------------------------------------
# Geometry of a workload (the oracle's own derivation)
# ---------------------------------------------------------------------------
def fit_pitch(R, D, n_rows, d_w, alpha_m) -> float:
    return _load().or_fit_pitch(R, D, n_rows, d_w, alpha_m)


def derive_geometry(cfg: dict) -> dict:
    """Full geometry of a workload from its primary parameters.

    Detector: columns span the fan of a square volume of half-width
    ``det_half_width`` (``n_cols_full`` columns, every ``col_keep``-th kept);
    rows are one voxel high at the isocentre (d_w = dz D / R).  Pitch: the
    largest whose TD window fits the rows, times ``pitch_factor``, rounded down
    to a whole number of slices.  The volume is centred in the scan.
    """
    R, D, vox = float(cfg["R"]), float(cfg["D"]), float(cfg["voxel"])
    nx, ny, nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    g = dict(R=R, D=D, lambda0=0.0, z0=0.0, lambda_first=0.0,
             views_per_turn=int(cfg["views_per_turn"]),
             n_views=int(cfg["views_per_turn"]) * int(cfg["turns"]),
             n_rows=int(cfg["n_rows"]), n_cols=int(cfg["n_cols"]),
             alpha_offset=0.0, w_offset=0.0, nx=nx, ny=ny, nz=nz, dx=vox, dy=vox, dz=vox,
             x0=-0.5 * (nx - 1) * vox, y0=-0.5 * (ny - 1) * vox,
             n_psi=int(cfg.get("n_psi", 2 * int(cfg["n_rows"]))), endpoint_mode=int(cfg.get("endpoint_mode", 0)))
    a_det = math.asin(math.sqrt(2.0) * float(cfg["det_half_width"]) / R)
    g["d_alpha"] = 2.0 * a_det / (int(cfg["n_cols_full"]) - 1) * int(cfg["col_keep"])
    g["d_w"] = vox * D / R
    g["P"] = 1.0  # placeholder for the alpha_m call (alpha_m does not use P)
    g["z_first"] = 0.0
    alpha_m = _load().or_alpha_m(ctypes.byref(_g(g)))
    pmax = fit_pitch(R, D, g["n_rows"], g["d_w"], alpha_m)
    g["P"] = math.floor(float(cfg["pitch_factor"]) * pmax / vox) * vox
    dl = 2.0 * math.pi / g["views_per_turn"]
    zc = g["z0"] + g["P"] / (2.0 * math.pi) * (g["lambda_first"] + 0.5 * g["n_views"] * dl)
    g["z_first"] = zc - 0.5 * (nz - 1) * vox
    return g


# ---------------------------------------------------------------------------
# Scalar functions
# ---------------------------------------------------------------------------
def r_fov(geom):
    return _load().or_r_fov(ctypes.byref(_g(geom)))


def alpha_m(geom):
    return _load().or_alpha_m(ctypes.byref(_g(geom)))


def w_kappa(geom, alpha, psi):
    return _load().or_w_kappa(ctypes.byref(_g(geom)), alpha, psi)


def w_td_top(geom, alpha):
    return _load().or_w_td_top(ctypes.byref(_g(geom)), alpha)


def w_td_bottom(geom, alpha):
    return _load().or_w_td_bottom(ctypes.byref(_g(geom)), alpha)


def psi_hat(geom, alpha, w):
    out = ctypes.c_double()
    ok = _load().or_psi_hat(ctypes.byref(_g(geom)), alpha, w, ctypes.byref(out))
    return out.value if ok else None


def pi_endpoints(geom, x, y, z):
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().or_pi_endpoints(ctypes.byref(_g(geom)), x, y, z, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def project_point(geom, lam, x, y, z):
    a, w, v = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().or_project_point(ctypes.byref(_g(geom)), lam, x, y, z, ctypes.byref(a), ctypes.byref(w),
                             ctypes.byref(v))
    return a.value, w.value, v.value


def n_psi(geom):
    return geom["n_psi"] if geom["n_psi"] > 0 else 2 * geom["n_rows"]


def pitch_slices(geom):
    return int(round(geom["P"] / geom["dz"]))


# ---------------------------------------------------------------------------
# Tables
# ---------------------------------------------------------------------------
def kappa_table(geom):
    g = _g(geom)
    idx = np.empty((n_psi(geom), geom["n_cols"] - 1), np.int32)
    frac = np.empty(idx.shape, np.float64)
    _load().or_kappa_table(ctypes.byref(g), _p(idx), _p(frac))
    return idx, frac


def psi_table(geom):
    g = _g(geom)
    idx = np.empty((geom["n_rows"], geom["n_cols"]), np.int32)
    frac = np.empty(idx.shape, np.float64)
    _load().or_psi_table(ctypes.byref(g), _p(idx), _p(frac))
    return idx, frac


def pi_table(geom):
    g = _g(geom)
    shape = (pitch_slices(geom), geom["ny"], geom["nx"])
    k0 = np.empty(shape, np.int32)
    k1 = np.empty(shape, np.int32)
    w0 = np.empty(shape)
    w1 = np.empty(shape)
    li = np.empty(shape)
    lo = np.empty(shape)
    _load().or_pi_table(ctypes.byref(g), _p(k0), _p(k1), _p(w0), _p(w1), _p(li), _p(lo))
    return dict(k0=k0, k1=k1, w0=w0, w1=w1, lam_i=li, lam_o=lo)


# ---------------------------------------------------------------------------
# Steps
# ---------------------------------------------------------------------------
def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def derivative(geom, sino):
    s = _f64(sino)
    out = np.empty((s.shape[0] - 1, geom["n_rows"], geom["n_cols"] - 1))
    _load().or_derivative(ctypes.byref(_g(geom)), _p(s), s.shape[0], _p(out))
    return out


def length_weight(geom, g1):
    out = _f64(g1).copy()
    _load().or_length_weight(ctypes.byref(_g(geom)), _p(out), out.shape[0])
    return out


def forward_rebin(geom, kap, g2):
    idx, frac = kap
    a = _f64(g2)
    out = np.empty((a.shape[0], n_psi(geom), geom["n_cols"] - 1))
    _load().or_forward_rebin(ctypes.byref(_g(geom)), _p(idx), _p(frac), _p(a), a.shape[0], _p(out))
    return out


def hilbert(geom, g3):
    a = _f64(g3)
    out = np.empty((a.shape[0], a.shape[1], geom["n_cols"]))
    gg = dict(geom)
    gg["n_psi"] = a.shape[1]
    _load().or_hilbert(ctypes.byref(_g(gg)), _p(a), a.shape[0], _p(out))
    return out


def backward_rebin(geom, psit, g4):
    idx, frac = psit
    a = _f64(g4)
    out = np.empty((a.shape[0], geom["n_rows"], geom["n_cols"]))
    _load().or_backward_rebin(ctypes.byref(_g(geom)), _p(idx), _p(frac), _p(a), a.shape[0], _p(out))
    return out


def post_cosine(geom, g5):
    out = _f64(g5).copy()
    _load().or_post_cosine(ctypes.byref(_g(geom)), _p(out), out.shape[0])
    return out


class Plan:
    """The oracle's pre-calculated tables for one geometry (one pitch)."""

    def __init__(self, geom: dict, with_pi: bool = True):
        self.geom = dict(geom)
        self.kap = kappa_table(geom)
        self.psi = psi_table(geom)
        self.pi = pi_table(geom) if with_pi else None

    # -- steps 1-6
    def filter(self, sino, v_begin: int = 0, n_out: int | None = None):
        """g^F for half-views [v_begin, v_begin + n_out) from sino[v_begin : v_begin + n_out + 1]."""
        s = np.asarray(sino)
        if n_out is None:
            n_out = s.shape[0] - 1 - v_begin
        part = _f64(s[v_begin:v_begin + n_out + 1])
        out = np.empty((n_out, self.geom["n_rows"], self.geom["n_cols"]))
        _load().or_filter(ctypes.byref(_g(self.geom)), _p(self.kap[0]), _p(self.kap[1]),
                          _p(self.psi[0]), _p(self.psi[1]), _p(part), part.shape[0], _p(out))
        return out

    # -- step 7
    def backproject(self, gF, gf_v0: int = 0):
        a = _f64(gF)
        vol = np.empty((self.geom["nz"], self.geom["ny"], self.geom["nx"]))
        t = self.pi
        rc = _load().or_backproject(ctypes.byref(_g(self.geom)), _p(t["k0"]), _p(t["k1"]), _p(t["w0"]),
                                    _p(t["w1"]), _p(a), gf_v0, a.shape[0], _p(vol))
        if rc != 0:
            raise ValueError("filtered views do not cover every voxel's PI window")
        return vol

    def recon(self, sino):
        return self.backproject(self.filter(sino), 0)

    # -- transposes
    def backproject_adjoint(self, vol, gf_v0: int, gf_nv: int):
        v = _f64(vol)
        out = np.empty((gf_nv, self.geom["n_rows"], self.geom["n_cols"]))
        t = self.pi
        rc = _load().or_backproject_adjoint(ctypes.byref(_g(self.geom)), _p(t["k0"]), _p(t["k1"]),
                                            _p(t["w0"]), _p(t["w1"]), _p(v), _p(out), gf_v0, gf_nv)
        if rc != 0:
            raise ValueError("filtered views do not cover every voxel's PI window")
        return out

    def filter_adjoint(self, gF):
        a = _f64(gF)
        out = np.empty((a.shape[0] + 1, self.geom["n_rows"], self.geom["n_cols"]))
        _load().or_filter_adjoint(ctypes.byref(_g(self.geom)), _p(self.kap[0]), _p(self.kap[1]),
                                  _p(self.psi[0]), _p(self.psi[1]), _p(a), a.shape[0], _p(out))
        return out

    def adjoint(self, vol):
        """Transpose of recon: volume -> sinogram of n_views views."""
        nv = self.geom["n_views"] - 1
        return self.filter_adjoint(self.backproject_adjoint(vol, 0, nv))

    def extents(self):
        out = np.empty(6)
        t = self.pi
        _load().or_extents(ctypes.byref(_g(self.geom)), _p(t["k0"]), _p(t["k1"]), _p(t["lam_i"]),
                           _p(t["lam_o"]), _p(out))
        return out

    def update_count(self):
        t = self.pi
        return int(_load().or_update_count(ctypes.byref(_g(self.geom)), _p(t["k0"]), _p(t["k1"])))


# ---------------------------------------------------------------------------
# Sampled backprojection (full-size workloads)
# ---------------------------------------------------------------------------
def pi_windows(geom, ijk):
    p = np.ascontiguousarray(ijk, dtype=np.int64).reshape(-1, 3)
    n = p.shape[0]
    ka = np.empty(n, np.int64)
    kb = np.empty(n, np.int64)
    wa = np.empty(n)
    wb = np.empty(n)
    _load().or_pi_window_points(ctypes.byref(_g(geom)), n, _p(p), _p(ka), _p(kb), _p(wa), _p(wb))
    return ka, kb, wa, wb


def backproject_points(geom, gF, gf_v0, ijk, windows=None):
    p = np.ascontiguousarray(ijk, dtype=np.int64).reshape(-1, 3)
    ka, kb, wa, wb = windows if windows is not None else pi_windows(geom, p)
    a = _f64(gF)
    out = np.empty(p.shape[0])
    rc = _load().or_backproject_points(ctypes.byref(_g(geom)), _p(a), gf_v0, a.shape[0], p.shape[0], _p(p),
                                       _p(ka), _p(kb), _p(wa), _p(wb), _p(out))
    if rc != 0:
        raise ValueError("filtered views do not cover a sampled voxel's PI window")
    return out


# ---------------------------------------------------------------------------
# Data simulation (the paper's Sec. III-C data generation)
# ---------------------------------------------------------------------------
def ray(geom, k, r, c):
    """Source point a and direction d (a + d is the detector sample) of view k, row r, column c."""
    a, d = np.zeros(3), np.zeros(3)
    _load().or_ray(ctypes.byref(_g(geom)), k, r, c, _p(a), _p(d))
    return a, d


def project(geom, vol, v0=0, nv=None):
    """Line integrals of the voxel function (cubes of constant value) for views v0 .. v0+nv-1."""
    nv = geom["n_views"] - v0 if nv is None else nv
    f = _f64(vol)
    out = np.empty((nv, geom["n_rows"], geom["n_cols"]))
    _load().or_project(ctypes.byref(_g(geom)), _p(f), v0, nv, _p(out))
    return out


def sparse_upsample(geom, sino, keep):
    """Keep every keep-th detector column, interpolate linearly back to all columns."""
    s = _f64(sino)
    out = np.empty_like(s)
    _load().or_sparse_upsample(ctypes.byref(_g(geom)), _p(s), s.shape[0], keep, _p(out))
    return out


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _load().or_philox4x32_10(c, k, o)
    return list(o)


def poisson(lam, seed, i):
    return _load().or_poisson(lam, seed, i)


def gaussian(seed, i):
    return _load().or_gaussian(seed, i)


def add_noise(g_up, I0=1e5, mean=0.0, var=0.5, seed=0):
    """(g_in, Poisson counts, M) of the Gaussian+Poisson model applied to g_up."""
    a = _f64(g_up)
    out = np.empty_like(a)
    counts = np.empty(a.shape, np.int64)
    M = ctypes.c_double()
    _load().or_add_noise(_p(a), a.size, I0, mean, var, seed, _p(out), _p(counts), ctypes.byref(M))
    return out, counts, M.value
