"""ctypes binding of libkatsevich.so: the C-ABI entry points under the same
names, argument marshalling only.  Every step of the operator runs in the
library's CUDA kernels; nothing here computes on the host."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# KATSEVICH_DEBUG_CHECKS=1 loads the bounds-checked build (paper_2201_02309_b300.build.build(debug=True))
LIB_PATH = os.path.join(HERE, "_lib", "libkatsevich_debug.so" if os.environ.get("KATSEVICH_DEBUG_CHECKS") == "1"
                        else "libkatsevich.so")

KATS_OK, KATS_EINVAL, KATS_EGEOM, KATS_ENOMEM, KATS_ECUDA, KATS_ETIMEOUT, KATS_ESPACE = range(7)
KATS_PREC_FP32, KATS_PREC_BF16, KATS_PREC_FP16 = 0, 1, 2
KATS_ENDPOINT_FRACTIONAL, KATS_ENDPOINT_HARD = 0, 1

_STATUS = {1: "KATS_EINVAL", 2: "KATS_EGEOM", 3: "KATS_ENOMEM", 4: "KATS_ECUDA", 5: "KATS_ETIMEOUT", 6: "KATS_ESPACE"}

# Every symbol include/katsevich.h declares.
EXPORTS = ["katsevich_fit_pitch", "katsevich_plan", "katsevich_plan_info", "katsevich_workspace_bytes",
           "katsevich_recon", "katsevich_adjoint", "katsevich_filter", "katsevich_backproject",
           "katsevich_host_workspace_bytes", "katsevich_recon_host", "katsevich_slab_views",
           "katsevich_recon_slab", "katsevich_plan_table",
           "katsevich_pi_endpoints", "katsevich_plan_destroy", "katsevich_last_error",
           "katsevich_recon_noalloc", "katsevich_device_status", "katsevich_backproject_adjoint",
           "katsevich_filter_adjoint", "katsevich_server_create", "katsevich_server_submit",
           "katsevich_server_wait", "katsevich_server_stats", "katsevich_server_destroy",
           "katsevich_arena_create", "katsevich_arena_alloc", "katsevich_arena_free",
           "katsevich_arena_largest_free", "katsevich_arena_in_use", "katsevich_arena_destroy",
           "katsevich_debug_fail_allocs", "katsevich_project", "katsevich_sparse_upsample",
           "katsevich_noise_workspace_bytes", "katsevich_add_noise", "katsevich_smem_read_bandwidth",
           "katsevich_tex_bilinear_rate",
           "katsevich_launch_count", "katsevich_debug_checks_enabled", "katsevich_debug_check_flags",
           "katsevich_debug_narrow_window", "katsevich_debug_nonmonotone", "katsevich_debug_wait_limit",
           "katsevich_debug_stall_producer", "katsevich_slice_groups"]


I32P = ctypes.POINTER(ctypes.c_int32)


class kats_geometry(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("D", ctypes.c_double), ("P", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("z0", ctypes.c_double), ("lambda_first", ctypes.c_double),
                ("views_per_turn", ctypes.c_int64), ("n_views", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("d_alpha", ctypes.c_double), ("alpha_offset", ctypes.c_double),
                ("d_w", ctypes.c_double), ("w_offset", ctypes.c_double),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z_first", ctypes.c_double),
                ("n_psi", ctypes.c_int64), ("endpoint_mode", ctypes.c_int64), ("flags", ctypes.c_int64)]


class kats_plan_info(ctypes.Structure):
    _fields_ = [("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("w_min", ctypes.c_double), ("w_max", ctypes.c_double),
                ("alpha_m", ctypes.c_double), ("psi_max", ctypes.c_double),
                ("slices_per_pitch", ctypes.c_int64), ("n_psi", ctypes.c_int64),
                ("first_view", ctypes.c_int64), ("n_filtered_views", ctypes.c_int64),
                ("update_count", ctypes.c_int64), ("gf_cols", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("plan_bytes", ctypes.c_int64), ("pi_monotone", ctypes.c_int64)]


class kats_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_int64), ("plan_cache_bytes", ctypes.c_int64),
                ("slots", ctypes.c_int32), ("max_bypass", ctypes.c_int32)]


class kats_request_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("plan_hit", ctypes.c_int32),
                ("bypassed", ctypes.c_int32), ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("gpu_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class kats_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "refused", "plan_hits",
                                              "plan_misses", "plan_evictions", "plans_cached", "arena_bytes",
                                              "arena_in_use_bytes", "arena_peak_bytes", "plan_cache_used_bytes")] + \
        [(n, ctypes.c_int32) for n in ("slots", "max_running", "pending", "running")]


class KatsevichError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree CUDA library; fail loudly when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libkatsevich.so is missing at {LIB_PATH}; run paper_2201_02309_b300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    sig = {
        "katsevich_fit_pitch": (ctypes.c_int, [ctypes.POINTER(kats_geometry), ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double)]),
        "katsevich_plan": (ctypes.c_int, [ctypes.POINTER(kats_geometry), ctypes.POINTER(P)]),
        "katsevich_plan_info": (ctypes.c_int, [P, ctypes.POINTER(kats_plan_info)]),
        "katsevich_workspace_bytes": (ctypes.c_int64, [P, ctypes.c_int]),
        "katsevich_recon": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_adjoint": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_filter": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_backproject": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
        "katsevich_host_workspace_bytes": (ctypes.c_int64, [P, ctypes.c_int, ctypes.c_int]),
        "katsevich_recon_host": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_slab_views": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64)]),
        "katsevich_recon_slab": (ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                P, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_plan_table": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_size_t]),
        "katsevich_pi_endpoints": (ctypes.c_int, [ctypes.POINTER(kats_geometry), ctypes.c_int64, P, P, P]),
        "katsevich_plan_destroy": (None, [P]),
        "katsevich_recon_noalloc": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
        "katsevich_smem_read_bandwidth": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
        "katsevich_tex_bilinear_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "katsevich_launch_count": (ctypes.c_int64, []),
        "katsevich_debug_checks_enabled": (ctypes.c_int, []),
        "katsevich_debug_check_flags": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
        "katsevich_debug_narrow_window": (None, [ctypes.c_int]),
        "katsevich_debug_nonmonotone": (None, [ctypes.c_int]),
        "katsevich_debug_wait_limit": (ctypes.c_int, [ctypes.c_int]),
        "katsevich_debug_stall_producer": (ctypes.c_int, [ctypes.c_int]),
        "katsevich_device_status": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
        "katsevich_backproject_adjoint": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
        "katsevich_filter_adjoint": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]),
        "katsevich_last_error": (ctypes.c_char_p, []),
        "katsevich_server_create": (ctypes.c_int, [ctypes.POINTER(kats_server_config), ctypes.POINTER(P)]),
        "katsevich_server_submit": (ctypes.c_int, [P, ctypes.POINTER(kats_geometry), P, P, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_uint64)]),
        "katsevich_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_int64,
                                                 ctypes.POINTER(kats_request_stats)]),
        "katsevich_server_stats": (ctypes.c_int, [P, ctypes.POINTER(kats_server_stats)]),
        "katsevich_server_destroy": (None, [P]),
        "katsevich_arena_create": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(P)]),
        "katsevich_arena_alloc": (ctypes.c_int64, [P, ctypes.c_int64]),
        "katsevich_arena_free": (ctypes.c_int, [P, ctypes.c_int64]),
        "katsevich_arena_largest_free": (ctypes.c_int64, [P]),
        "katsevich_arena_in_use": (ctypes.c_int64, [P]),
        "katsevich_arena_destroy": (None, [P]),
        "katsevich_debug_fail_allocs": (None, [ctypes.c_int]),
        "katsevich_slice_groups": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                  ctypes.c_int64, I32P, I32P, I32P, I32P, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int), I32P, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int)]),
        "katsevich_project": (ctypes.c_int, [ctypes.POINTER(kats_geometry), P, P, ctypes.c_int64, ctypes.c_int64,
                                             P]),
        "katsevich_sparse_upsample": (ctypes.c_int, [ctypes.POINTER(kats_geometry), P, P, ctypes.c_int64,
                                                     ctypes.c_int, P]),
        "katsevich_noise_workspace_bytes": (ctypes.c_int64, []),
        "katsevich_add_noise": (ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_uint64, P, P, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_double), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != KATS_OK:
        msg = load().katsevich_last_error().decode(errors="replace")
        raise KatsevichError(status, msg)


def geometry_struct(geom: dict) -> kats_geometry:
    vals = {k: geom.get(k, 0) for k, _ in kats_geometry._fields_}
    return kats_geometry(**vals)


# --- same names as the C ABI -------------------------------------------------
def katsevich_fit_pitch(geom: dict, factor: float = 1.0) -> float:
    out = ctypes.c_double()
    g = geometry_struct(geom)
    check(load().katsevich_fit_pitch(ctypes.byref(g), factor, ctypes.byref(out)))
    return out.value


def katsevich_plan(geom: dict) -> int:
    g = geometry_struct(geom)
    h = ctypes.c_void_p()
    check(load().katsevich_plan(ctypes.byref(g), ctypes.byref(h)))
    return h.value


def katsevich_plan_info(plan: int) -> dict:
    info = kats_plan_info()
    check(load().katsevich_plan_info(plan, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in kats_plan_info._fields_}


def katsevich_workspace_bytes(plan: int, precision: int = KATS_PREC_FP32) -> int:
    n = load().katsevich_workspace_bytes(plan, precision)
    if n < 0:
        raise KatsevichError(KATS_EINVAL, "workspace size unavailable for this precision")
    return n


def katsevich_recon(plan, sino_ptr, vol_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr) -> None:
    check(load().katsevich_recon(plan, sino_ptr, vol_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr))


def katsevich_adjoint(plan, vol_ptr, sino_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr) -> None:
    check(load().katsevich_adjoint(plan, vol_ptr, sino_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr))


def katsevich_filter(plan, sino_ptr, gF_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr) -> None:
    check(load().katsevich_filter(plan, sino_ptr, gF_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr))


def katsevich_backproject(plan, gF_ptr, vol_ptr, batch, stream_ptr) -> None:
    check(load().katsevich_backproject(plan, gF_ptr, vol_ptr, batch, stream_ptr))


def katsevich_backproject_adjoint(plan, vol_ptr, gF_ptr, batch, stream_ptr) -> None:
    check(load().katsevich_backproject_adjoint(plan, vol_ptr, gF_ptr, batch, stream_ptr))


def katsevich_filter_adjoint(plan, gF_ptr, sino_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr) -> None:
    check(load().katsevich_filter_adjoint(plan, gF_ptr, sino_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr))


def katsevich_host_workspace_bytes(plan, batch, precision=KATS_PREC_FP32) -> int:
    n = load().katsevich_host_workspace_bytes(plan, batch, precision)
    if n < 0:
        raise KatsevichError(KATS_EINVAL, "host workspace size unavailable")
    return n


def katsevich_recon_host(plan, host_sino_ptr, host_vol_ptr, batch, precision, ws_ptr, ws_bytes, stream_ptr) -> None:
    check(load().katsevich_recon_host(plan, host_sino_ptr, host_vol_ptr, batch, precision, ws_ptr, ws_bytes,
                                      stream_ptr))


def katsevich_slab_views(plan, s_begin, s_end) -> tuple:
    """(view_begin, view_count): the sinogram views slices [s_begin, s_end) read."""
    vb, vc = ctypes.c_int64(), ctypes.c_int64()
    check(load().katsevich_slab_views(plan, s_begin, s_end, ctypes.byref(vb), ctypes.byref(vc)))
    return vb.value, vc.value


def katsevich_recon_slab(plan, sino_ptr, view_begin, view_count, s_begin, s_end, vol_ptr, precision, ws_ptr,
                         ws_bytes, stream_ptr) -> None:
    check(load().katsevich_recon_slab(plan, sino_ptr, view_begin, view_count, s_begin, s_end, vol_ptr, precision,
                                      ws_ptr, ws_bytes, stream_ptr))


def katsevich_plan_table(plan, which, dst_ptr, nbytes) -> None:
    check(load().katsevich_plan_table(plan, which, dst_ptr, nbytes))


def katsevich_pi_endpoints(geom: dict, n, xyz_ptr, li_ptr, lo_ptr) -> None:
    g = geometry_struct(geom)
    check(load().katsevich_pi_endpoints(ctypes.byref(g), n, xyz_ptr, li_ptr, lo_ptr))


def katsevich_recon_noalloc(plan, sino_ptr, vol_ptr, batch, stream_ptr) -> None:
    check(load().katsevich_recon_noalloc(plan, sino_ptr, vol_ptr, batch, stream_ptr))


def katsevich_smem_read_bandwidth() -> float:
    """Measured shared-memory read bandwidth of the current GPU, bytes per second."""
    out = ctypes.c_double(0.0)
    check(load().katsevich_smem_read_bandwidth(ctypes.byref(out)))
    return out.value


def katsevich_tex_bilinear_rate(half_texels: bool = False) -> float:
    """Measured bilinear texture-fetch rate of the current GPU, samples per second."""
    out = ctypes.c_double(0.0)
    check(load().katsevich_tex_bilinear_rate(1 if half_texels else 0, ctypes.byref(out)))
    return out.value


def katsevich_launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(load().katsevich_launch_count())


def katsevich_debug_checks_enabled() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(load().katsevich_debug_checks_enabled())


def katsevich_debug_check_flags() -> int:
    """Invariant-violation bits recorded by the bounds-checked build (read and cleared)."""
    out = ctypes.c_int(0)
    check(load().katsevich_debug_check_flags(ctypes.byref(out)))
    return out.value


def katsevich_debug_narrow_window(cols: int) -> None:
    """Checked build only: stage view windows `cols` columns too narrow (0 ends it)."""
    load().katsevich_debug_narrow_window(int(cols))


def katsevich_debug_nonmonotone(on: bool) -> None:
    """Checked build only: every view through the general end-weight path (False ends it)."""
    load().katsevich_debug_nonmonotone(1 if on else 0)


def katsevich_debug_wait_limit(polls: int) -> None:
    """Checked build only: the staged backprojection's waits give up after `polls` polls (0: default)."""
    check(load().katsevich_debug_wait_limit(int(polls)))


def katsevich_debug_stall_producer(pairs: int) -> None:
    """Checked build only: its producer stops issuing after `pairs` view pairs (-1 ends it)."""
    check(load().katsevich_debug_stall_producer(int(pairs)))


def katsevich_device_status(plan) -> int:
    st = ctypes.c_int()
    check(load().katsevich_device_status(plan, ctypes.byref(st)))
    return st.value


def katsevich_plan_destroy(plan) -> None:
    load().katsevich_plan_destroy(plan)


def katsevich_last_error() -> str:
    return load().katsevich_last_error().decode(errors="replace")


# --- serving loop ------------------------------------------------------------
def katsevich_server_create(arena_bytes: int, plan_cache_bytes: int, slots: int, max_bypass: int = 8) -> int:
    cfg = kats_server_config(arena_bytes, plan_cache_bytes, slots, max_bypass)
    h = ctypes.c_void_p()
    check(load().katsevich_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def katsevich_server_submit(server: int, geom: dict, host_sino_ptr: int, host_vol_ptr: int,
                            precision: int = KATS_PREC_FP32) -> int:
    g = geometry_struct(geom)
    t = ctypes.c_uint64()
    check(load().katsevich_server_submit(server, ctypes.byref(g), host_sino_ptr, host_vol_ptr, precision,
                                         ctypes.byref(t)))
    return t.value


def katsevich_server_wait(server: int, ticket: int, timeout_ms: int):
    """(status, stats dict, message): the request's own status is returned, not raised."""
    st = kats_request_stats()
    rc = load().katsevich_server_wait(server, ticket, timeout_ms, ctypes.byref(st))
    msg = load().katsevich_last_error().decode(errors="replace") if rc else ""
    return rc, {k: getattr(st, k) for k, _ in kats_request_stats._fields_}, msg


def katsevich_server_stats(server: int) -> dict:
    st = kats_server_stats()
    check(load().katsevich_server_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in kats_server_stats._fields_}


def katsevich_server_destroy(server: int) -> None:
    load().katsevich_server_destroy(server)


def katsevich_arena_create(nbytes: int) -> int:
    h = ctypes.c_void_p()
    check(load().katsevich_arena_create(nbytes, ctypes.byref(h)))
    return h.value


def katsevich_arena_alloc(arena: int, nbytes: int) -> int:
    return load().katsevich_arena_alloc(arena, nbytes)


def katsevich_arena_free(arena: int, offset: int) -> None:
    check(load().katsevich_arena_free(arena, offset))


def katsevich_arena_largest_free(arena: int) -> int:
    return load().katsevich_arena_largest_free(arena)


def katsevich_arena_in_use(arena: int) -> int:
    return load().katsevich_arena_in_use(arena)


def katsevich_arena_destroy(arena: int) -> None:
    load().katsevich_arena_destroy(arena)


def katsevich_debug_fail_allocs(n: int) -> None:
    load().katsevich_debug_fail_allocs(n)


def katsevich_slice_groups(s_begin: int, s_end: int, slices_per_pitch: int, max_groups: int = 4,
                           lead_end: int = 2 ** 63 - 1):
    """The backprojection's slice grouping (host only): ([(groups, t, s0, cnt), ...], [(s, e), ...])."""
    cap = 4096
    arr = [(ctypes.c_int32 * cap)() for _ in range(4)]
    rest = (ctypes.c_int32 * (2 * cap))()
    ni, nr = ctypes.c_int(0), ctypes.c_int(0)
    check(load().katsevich_slice_groups(s_begin, s_end, slices_per_pitch, max_groups, lead_end, *arr, cap,
                                        ctypes.byref(ni), rest, cap, ctypes.byref(nr)))
    items = [tuple(int(a[i]) for a in arr) for i in range(ni.value)]
    return items, [(int(rest[2 * j]), int(rest[2 * j + 1])) for j in range(nr.value)]


# --- data simulation -----------------------------------------------------------
def katsevich_project(geom: dict, vol_ptr: int, sino_ptr: int, v0: int, nv: int, stream_ptr) -> None:
    g = geometry_struct(geom)
    check(load().katsevich_project(ctypes.byref(g), vol_ptr, sino_ptr, v0, nv, stream_ptr))


def katsevich_sparse_upsample(geom: dict, sino_ptr: int, out_ptr: int, nv: int, keep: int, stream_ptr) -> None:
    g = geometry_struct(geom)
    check(load().katsevich_sparse_upsample(ctypes.byref(g), sino_ptr, out_ptr, nv, keep, stream_ptr))


def katsevich_noise_workspace_bytes() -> int:
    return load().katsevich_noise_workspace_bytes()


def katsevich_add_noise(g_up_ptr, g_in_ptr, n, I0, mean, var, seed, counts_ptr, ws_ptr, ws_bytes, stream_ptr,
                        want_M: bool = True):
    M = ctypes.c_double()
    check(load().katsevich_add_noise(g_up_ptr, g_in_ptr, n, I0, mean, var, seed, counts_ptr, ws_ptr, ws_bytes,
                                     ctypes.byref(M) if want_M else None, stream_ptr))
    return M.value if want_M else None
