"""C-ABI library checks that need no GPU: it loads, exports every symbol the
public header declares, and its host-only logic matches the oracle."""
import math
import os
import re

import pytest

import oracle
import synth
from paper_2201_02309_b300 import build as pkg_build
from paper_2201_02309_b300 import make_geometry, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return native.load()


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"KATS_API[^;(]*?\b(katsevich_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(native.EXPORTS) == names


def test_fit_pitch_and_geometry_match_oracle(lib):
    for ci in (1, 2, 3, 4):
        cfg = synth.config(ci)
        mine = make_geometry(cfg)
        ref = oracle.derive_geometry(cfg)
        for k in oracle.GEOM_KEYS:
            assert mine[k] == pytest.approx(ref[k], rel=1e-13, abs=1e-12), (ci, k)


def test_fit_pitch_closed_form(lib):
    g = make_geometry(synth.config(1))
    am = math.asin(32 * math.sqrt(2) / 500)
    h = 15.5 * 2.0 * 500 * math.cos(am) / (1000 * (math.pi / 2 + am))
    assert native.katsevich_fit_pitch(g, 1.0) == math.floor(2 * math.pi * h)
    assert native.katsevich_fit_pitch(g, 1.5) == math.floor(1.5 * 2 * math.pi * h)


@pytest.mark.parametrize("field,value", [("R", -1.0), ("P", 57.5), ("nx", 0), ("flags", 1), ("n_psi", 1),
                                         ("endpoint_mode", 7), ("d_w", 0.0), ("R", 40.0)])
def test_invalid_geometry_rejected_on_host(lib, field, value):
    g = make_geometry(synth.config(1))
    g[field] = value
    with pytest.raises(native.KatsevichError) as e:
        native.katsevich_plan(g)
    assert e.value.status == native.KATS_EGEOM
    assert native.katsevich_last_error()


def test_null_arguments(lib):
    import ctypes
    assert lib.katsevich_plan(None, None) == native.KATS_EINVAL
    assert lib.katsevich_recon(None, None, None, 1, 0, None, 0, None) == native.KATS_EINVAL
    assert lib.katsevich_plan_info(None, None) == native.KATS_EINVAL
    assert lib.katsevich_workspace_bytes(None, 0) == -1
    lib.katsevich_plan_destroy(None)
    h = ctypes.c_void_p()
    assert lib.katsevich_plan(None, ctypes.byref(h)) == native.KATS_EINVAL


def test_measurement_and_debug_entry_points_host_side(lib):
    """The measurement and checked-build entry points answer on the host: NULL outputs are
    KATS_EINVAL, the plain build reports no checks (narrowing is a no-op there), and the
    launch counter is a non-negative count."""
    assert lib.katsevich_smem_read_bandwidth(None) == native.KATS_EINVAL
    assert lib.katsevich_tex_bilinear_rate(0, None) == native.KATS_EINVAL
    assert lib.katsevich_debug_check_flags(None) == native.KATS_EINVAL
    assert native.katsevich_debug_checks_enabled() is False
    native.katsevich_debug_narrow_window(8)
    native.katsevich_debug_narrow_window(0)
    n0 = native.katsevich_launch_count()
    assert isinstance(n0, int) and n0 >= 0
    assert native.katsevich_launch_count() == n0  # nothing launched in between
