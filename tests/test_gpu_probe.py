"""The shared-memory read-bandwidth probe that grounds the backprojection's roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_smem_read_bandwidth_near_unit_count_peak():
    import torch
    import paper_2201_02309_b300.native as native

    props = torch.cuda.get_device_properties(0)
    bw = max(native.katsevich_smem_read_bandwidth() for _ in range(2))
    # 128 B per clock per SM at the maximum SM clock bounds it from above (a little slack for
    # timer granularity); half of it from below catches a probe that measures something else
    derived = props.multi_processor_count * 128 * 2032e6
    assert 0.5 * derived < bw < 1.05 * derived


def test_smem_read_bandwidth_rejects_null():
    import ctypes
    import paper_2201_02309_b300.native as native

    assert native.load().katsevich_smem_read_bandwidth(ctypes.POINTER(ctypes.c_double)()) == 1  # KATS_EINVAL


def test_launch_count_per_reconstruction():
    """One FP32 reconstruction is four launches: derivative + rebinning, the Hilbert
    contraction, backward rebinning + cosine, backprojection."""
    import torch

    import paper_2201_02309_b300 as kats
    import paper_2201_02309_b300.native as native
    import synth

    plan = kats.Plan(kats.make_geometry(synth.config(1)))
    sino = torch.rand(plan.sino_shape, device="cuda")
    plan.recon(sino)
    torch.cuda.synchronize()
    n0 = native.katsevich_launch_count()
    for _ in range(3):
        plan.recon(sino)
    torch.cuda.synchronize()
    assert native.katsevich_launch_count() - n0 == 12


def test_tex_bilinear_rate_plausible():
    import paper_2201_02309_b300.native as native

    for half in (False, True):
        r = native.katsevich_tex_bilinear_rate(half)
        # between one filtered sample per SM per 4 clocks and 64 per SM per clock at 2 GHz
        assert 148 * 0.25 * 1e9 < r < 148 * 64 * 2.1e9, (half, r)
