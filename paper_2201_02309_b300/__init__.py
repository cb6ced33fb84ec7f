"""B300-native Katsevich helical cone-beam reconstruction (curved detector,
pitch by pitch) behind a C-ABI CUDA library.

``Plan`` wraps one geometry's device-resident tables; ``Plan.recon`` runs
steps 1-7 of the paper's Section II on torch CUDA tensors, ``Plan.adjoint`` its
exact transpose.  PyTorch provides device memory and streams only; the
arithmetic is in ``csrc/*.cu``.  There is no CPU fallback: without the built
library or a CUDA device every call raises.
"""
from __future__ import annotations

import math

import numpy as np

from . import native
from .native import (KATS_ENDPOINT_FRACTIONAL, KATS_ENDPOINT_HARD, KATS_PREC_BF16, KATS_PREC_FP16,  # noqa: F401
                     KATS_PREC_FP32, KatsevichError)

__all__ = ["Plan", "make_geometry", "slab_partition", "KatsevichError", "native"]


def make_geometry(cfg: dict) -> dict:
    """Geometry of a workload from its primary parameters.

    Detector columns span the fan of a square volume of half-width
    ``det_half_width`` (``n_cols_full`` columns, every ``col_keep``-th kept),
    rows are one voxel high at the isocentre (d_w = dz D / R), the pitch is the
    largest whose Tam-Danielsson window fits the rows times ``pitch_factor``
    (``katsevich_fit_pitch``), and the volume is centred in the scan.
    """
    R, D, vox = float(cfg["R"]), float(cfg["D"]), float(cfg["voxel"])
    nx, ny, nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    vpt = int(cfg["views_per_turn"])
    g = dict(R=R, D=D, P=0.0, lambda0=0.0, z0=0.0, lambda_first=0.0, views_per_turn=vpt,
             n_views=vpt * int(cfg["turns"]), n_rows=int(cfg["n_rows"]), n_cols=int(cfg["n_cols"]),
             alpha_offset=0.0, w_offset=0.0, nx=nx, ny=ny, nz=nz, dx=vox, dy=vox, dz=vox,
             x0=-0.5 * (nx - 1) * vox, y0=-0.5 * (ny - 1) * vox, z_first=0.0,
             n_psi=int(cfg.get("n_psi", 2 * int(cfg["n_rows"]))),
             endpoint_mode=int(cfg.get("endpoint_mode", 0)), flags=0)
    half_fan = math.asin(math.sqrt(2.0) * float(cfg["det_half_width"]) / R)
    g["d_alpha"] = 2.0 * half_fan / (int(cfg["n_cols_full"]) - 1) * int(cfg["col_keep"])
    g["d_w"] = vox * D / R
    g["P"] = native.katsevich_fit_pitch(g, float(cfg["pitch_factor"]))
    dl = 2.0 * math.pi / vpt
    zc = g["z0"] + g["P"] / (2.0 * math.pi) * (g["lambda_first"] + 0.5 * g["n_views"] * dl)
    g["z_first"] = zc - 0.5 * (nz - 1) * vox
    return g


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2201_02309_b300 needs a CUDA device (no CPU fallback)")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """Device-resident pre-calculated tables of one geometry (one pitch)."""

    TABLES = {"kappa_idx": (0, np.int32, "kappa"), "kappa_frac": (1, np.float32, "kappa"),
              "psi_idx": (2, np.int32, "psi"), "psi_frac": (3, np.float32, "psi"),
              "k0": (4, np.int32, "pi"), "k1": (5, np.int32, "pi"),
              "w0": (6, np.float32, "pi"), "w1": (7, np.float32, "pi")}

    def __init__(self, geom: dict):
        _torch()
        self.geom = dict(geom)
        self.handle = native.katsevich_plan(self.geom)
        self.info = native.katsevich_plan_info(self.handle)
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            native.katsevich_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes
    @property
    def sino_shape(self):
        g = self.geom
        return (g["n_views"], g["n_rows"], g["n_cols"])

    @property
    def vol_shape(self):
        g = self.geom
        return (g["nz"], g["ny"], g["nx"])

    @property
    def filtered_shape(self):
        """[views][rows][gf_cols]: rows padded to a multiple of 4 floats, pad columns zero."""
        g = self.geom
        return (self.info["n_filtered_views"], g["n_rows"], self.info["gf_cols"])

    def workspace(self, precision=KATS_PREC_FP32, device=None):
        """A cached device workspace (torch uint8) big enough for recon/adjoint."""
        torch = _torch()
        n = native.katsevich_workspace_bytes(self.handle, precision)
        if self._ws is None or self._ws.numel() < n:
            self._ws = torch.empty(n, dtype=torch.uint8, device=device or "cuda")
        return self._ws

    # -- operator
    def _batch(self, x, item_shape):
        if x.dtype != _torch().float32 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if tuple(x.shape[-3:]) != tuple(item_shape):
            raise ValueError(f"expected trailing shape {item_shape}, got {tuple(x.shape)}")
        return 1 if x.dim() == 3 else int(np.prod(x.shape[:-3]))

    def recon(self, sino, out=None, precision=KATS_PREC_FP32, stream=None, workspace=None):
        torch = _torch()
        b = self._batch(sino, self.sino_shape)
        if out is None:
            out = torch.empty(sino.shape[:-3] + self.vol_shape, dtype=torch.float32, device=sino.device)
        ws = workspace if workspace is not None else self.workspace(precision, sino.device)
        native.katsevich_recon(self.handle, sino.data_ptr(), out.data_ptr(), b, precision, ws.data_ptr(),
                               ws.numel() * ws.element_size(), _stream_ptr(stream))
        return out

    def adjoint(self, vol, out=None, precision=KATS_PREC_FP32, stream=None, workspace=None):
        torch = _torch()
        b = self._batch(vol, self.vol_shape)
        if out is None:
            out = torch.empty(vol.shape[:-3] + self.sino_shape, dtype=torch.float32, device=vol.device)
        ws = workspace if workspace is not None else self.workspace(precision, vol.device)
        native.katsevich_adjoint(self.handle, vol.data_ptr(), out.data_ptr(), b, precision, ws.data_ptr(),
                                 ws.numel() * ws.element_size(), _stream_ptr(stream))
        return out

    def filter(self, sino, precision=KATS_PREC_FP32, stream=None):
        torch = _torch()
        b = self._batch(sino, self.sino_shape)
        out = torch.empty(sino.shape[:-3] + self.filtered_shape, dtype=torch.float32, device=sino.device)
        ws = self.workspace(precision, sino.device)
        native.katsevich_filter(self.handle, sino.data_ptr(), out.data_ptr(), b, precision, ws.data_ptr(),
                                ws.numel() * ws.element_size(), _stream_ptr(stream))
        return out

    def backproject(self, gF, stream=None):
        torch = _torch()
        b = self._batch(gF, self.filtered_shape)
        out = torch.empty(gF.shape[:-3] + self.vol_shape, dtype=torch.float32, device=gF.device)
        native.katsevich_backproject(self.handle, gF.data_ptr(), out.data_ptr(), b, _stream_ptr(stream))
        return out

    def backproject_adjoint(self, vol, stream=None):
        """Transpose of step 7: volume -> filtered-data layout [views][rows][gf_cols]."""
        torch = _torch()
        b = self._batch(vol, self.vol_shape)
        out = torch.empty(vol.shape[:-3] + self.filtered_shape, dtype=torch.float32, device=vol.device)
        native.katsevich_backproject_adjoint(self.handle, vol.data_ptr(), out.data_ptr(), b, _stream_ptr(stream))
        return out

    def filter_adjoint(self, gF, precision=KATS_PREC_FP32, stream=None):
        """Transpose of steps 1-6: filtered-data layout -> sinogram."""
        torch = _torch()
        b = self._batch(gF, self.filtered_shape)
        out = torch.empty(gF.shape[:-3] + self.sino_shape, dtype=torch.float32, device=gF.device)
        ws = self.workspace(precision, gF.device)
        native.katsevich_filter_adjoint(self.handle, gF.data_ptr(), out.data_ptr(), b, precision, ws.data_ptr(),
                                        ws.numel() * ws.element_size(), _stream_ptr(stream))
        return out

    def recon_host(self, host_sino, host_vol, batch=1, precision=KATS_PREC_FP32, stream=None, workspace=None):
        """End-to-end call on host (ideally pinned) torch CPU tensors; synchronous."""
        torch = _torch()
        n = native.katsevich_host_workspace_bytes(self.handle, batch, precision)
        if workspace is None or workspace.numel() < n:
            workspace = torch.empty(n, dtype=torch.uint8, device="cuda")
        native.katsevich_recon_host(self.handle, host_sino.data_ptr(), host_vol.data_ptr(), batch, precision,
                                    workspace.data_ptr(), n, _stream_ptr(stream))
        return host_vol

    # -- z-slab partition (one volume over several GPUs: one slab each, no exchange)
    def slab_views(self, s_begin: int, s_end: int):
        """(view_begin, view_count): the sinogram views slices [s_begin, s_end) read."""
        return native.katsevich_slab_views(self.handle, s_begin, s_end)

    def recon_slab(self, sino_views, view_begin: int, s_begin: int, s_end: int, out=None,
                   precision=KATS_PREC_FP32, stream=None, workspace=None):
        """Slices [s_begin, s_end) (s_begin a multiple of 16) from sinogram views
        [view_begin, view_begin + len(sino_views)); equal to those slices of recon() to FP32
        rounding (the backprojection groups slices one or more pitches apart within a launch, so a
        slab can group a slice differently from the whole volume)."""
        torch = _torch()
        g = self.geom
        if sino_views.dtype != torch.float32 or not sino_views.is_cuda or not sino_views.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor")
        if sino_views.dim() != 3 or tuple(sino_views.shape[1:]) != (g["n_rows"], g["n_cols"]):
            raise ValueError(f"expected [views][{g['n_rows']}][{g['n_cols']}], got {tuple(sino_views.shape)}")
        shape = (s_end - s_begin, g["ny"], g["nx"])
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=sino_views.device)
        elif tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous():
            raise ValueError(f"expected a contiguous float32 output of shape {shape}")
        ws = workspace if workspace is not None else self.workspace(precision, sino_views.device)
        native.katsevich_recon_slab(self.handle, sino_views.data_ptr(), view_begin, sino_views.shape[0], s_begin,
                                    s_end, out.data_ptr(), precision, ws.data_ptr(), ws.numel() * ws.element_size(),
                                    _stream_ptr(stream))
        return out

    # -- tables (for checks)
    def table(self, name: str) -> np.ndarray:
        which, dt, kind = self.TABLES[name]
        g = self.geom
        if kind == "kappa":
            shape = (self.info["n_psi"], g["n_cols"] - 1)
        elif kind == "psi":
            shape = (g["n_rows"], g["n_cols"])
        else:
            shape = (self.info["slices_per_pitch"], g["ny"], g["nx"])
        a = np.empty(shape, dt)
        native.katsevich_plan_table(self.handle, which, a.ctypes.data, a.nbytes)
        return a


def slab_partition(nz: int, world: int, tile: int = 16):
    """Contiguous slice ranges [(s_begin, s_end)] for `world` ranks: every start a
    multiple of `tile` (the backprojection's slice tile), tile counts as even as
    possible, earlier ranks taking the extra tiles; a rank left without a tile gets
    an empty range (s, s)."""
    if nz < 1 or world < 1 or tile < 1:
        raise ValueError("nz, world and tile must be >= 1")
    n_tiles = -(-nz // tile)
    out, t0 = [], 0
    for r in range(world):
        t1 = t0 + n_tiles // world + (1 if r < n_tiles % world else 0)
        out.append((min(t0 * tile, nz), min(t1 * tile, nz)))
        t0 = t1
    return out


def pi_endpoints(geom: dict, xyz: np.ndarray):
    """The device FP64 PI-line solver on host points (for checks)."""
    p = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    li = np.empty(p.shape[0])
    lo = np.empty(p.shape[0])
    native.katsevich_pi_endpoints(geom, p.shape[0], p.ctypes.data, li.ctypes.data, lo.ctypes.data)
    return li, lo


# --- data simulation (the paper's Sec. III-C data generation) ---------------------
def project(geom: dict, vol, v0: int = 0, nv: int | None = None, stream=None):
    """Helical projection of a float32 CUDA volume [nz][ny][nx]: line integrals of
    the voxel function for views v0 .. v0+nv-1 -> [nv][n_rows][n_cols]."""
    torch = _torch()
    nv = geom["n_views"] - v0 if nv is None else nv
    if vol.dtype != torch.float32 or not vol.is_cuda or not vol.is_contiguous() or \
            tuple(vol.shape) != (geom["nz"], geom["ny"], geom["nx"]):
        raise ValueError("expected a contiguous float32 CUDA volume [nz][ny][nx]")
    out = torch.empty((nv, geom["n_rows"], geom["n_cols"]), dtype=torch.float32, device=vol.device)
    native.katsevich_project(geom, vol.data_ptr(), out.data_ptr(), v0, nv, _stream_ptr(stream))
    return out


def sparse_upsample(geom: dict, sino, keep: int = 4, stream=None):
    """Keep every keep-th detector column, interpolate linearly back to all columns."""
    torch = _torch()
    if sino.dtype != torch.float32 or not sino.is_cuda or not sino.is_contiguous() or sino.shape[-1] != geom["n_cols"]:
        raise ValueError("expected a contiguous float32 CUDA sinogram [views][n_rows][n_cols]")
    out = torch.empty_like(sino)
    native.katsevich_sparse_upsample(geom, sino.data_ptr(), out.data_ptr(), sino.numel() // (geom["n_rows"] *
                                     geom["n_cols"]), keep, _stream_ptr(stream))
    return out


def add_noise(g_up, I0: float = 1e5, mean: float = 0.0, var: float = 0.5, seed: int = 0, return_counts=False,
              stream=None):
    """Gaussian+Poisson noise of the paper's data generation: (g_in, M[, counts])."""
    torch = _torch()
    if g_up.dtype != torch.float32 or not g_up.is_cuda or not g_up.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    out = torch.empty_like(g_up)
    counts = torch.empty(g_up.shape, dtype=torch.int64, device=g_up.device) if return_counts else None
    ws = torch.empty(native.katsevich_noise_workspace_bytes(), dtype=torch.uint8, device=g_up.device)
    M = native.katsevich_add_noise(g_up.data_ptr(), out.data_ptr(), g_up.numel(), I0, mean, var, seed,
                                   counts.data_ptr() if counts is not None else None, ws.data_ptr(), ws.numel(),
                                   _stream_ptr(stream))
    return (out, M, counts) if return_counts else (out, M)


def simulate_input(geom: dict, vol, keep: int = 4, I0: float = 1e5, var: float = 0.5, seed: int = 0, stream=None):
    """The network input of the paper's data generation: project the label
    volume, keep every keep-th column and upsample, add Gaussian+Poisson noise."""
    g_gt = project(geom, vol, stream=stream)
    g_up = sparse_upsample(geom, g_gt, keep, stream=stream) if keep > 1 else g_gt
    g_in, _ = add_noise(g_up, I0=I0, var=var, seed=seed, stream=stream)
    return g_gt, g_in
