"""Full-size parity: the 512 x 512 x 256 clinical workload (64 x 736 detector,
1160 views/turn, 8 turns) reconstructed on the GPU in the benchmark's launch
configuration, checked against the FP64 oracle on sampled voxels (PI windows
from the oracle's own PI-line solver, filtered views from the oracle's
filter on exactly the views those voxels need) and on sampled filtered views.
"""
import numpy as np
import pytest

import oracle
import synth
from cases import near_tie, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def c2():
    import torch

    import paper_2201_02309_b300 as kats
    cfg = synth.config(2)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(cfg, g, synth.phantom_seed(2))
    sino = synth.project(g, ell).astype(np.float32)
    kp = kats.Plan(g)
    dsino = torch.from_numpy(sino).cuda()
    vol = kp.recon(dsino)
    torch.cuda.synchronize()
    return g, sino, kp, dsino, vol.cpu().numpy()


def test_c2_plan_info_and_slabs(c2):
    g, sino, kp, _, _ = c2
    info = kp.info
    assert info["slices_per_pitch"] == 70 and g["P"] == 70.0
    # sampled columns of the one-pitch table vs the oracle's PI solver
    rng = np.random.default_rng(0)
    ijk = np.stack([rng.integers(0, 512, 3000), rng.integers(0, 512, 3000), rng.integers(0, 70, 3000)], 1)
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    k0, k1, w0, w1 = kp.table("k0"), kp.table("k1"), kp.table("w0"), kp.table("w1")
    i, j, s = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    bad0 = (k0[s, j, i] != ka) & ~near_tie(wa)
    bad1 = (k1[s, j, i] != kb) & ~near_tie(wb)
    assert not bad0.any() and not bad1.any()
    ok = k0[s, j, i] == ka
    assert np.abs(w0[s, j, i] - wa)[ok].max() < 2e-7


def test_c2_filtered_views_sampled(c2):
    import torch
    g, sino, kp, dsino, _ = c2
    gF = kp.filter(dsino)
    torch.cuda.synchronize()
    op = oracle.Plan(g, with_pi=False)
    v0 = kp.info["first_view"]
    for v in (0, 1777, kp.info["n_filtered_views"] - 1):
        want = op.filter(sino.astype(np.float64), v0 + v, 1)[0]
        assert rel_l2(gF[v, :, :g["n_cols"]].cpu().numpy(), want) < TOL


def test_c2_voxels_sampled(c2):
    g, sino, kp, _, vol = c2
    rng = np.random.default_rng(1)
    n = 240
    s = rng.integers(127, 130, n)
    ijk = np.stack([rng.integers(0, 512, n), rng.integers(0, 512, n), s], 1)
    # ragged corners and the volume edges of those slices
    ijk[:4, :2] = [(0, 0), (511, 0), (0, 511), (511, 511)]
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    v0, v1 = int(ka.min()), int(kb.max())
    op = oracle.Plan(g, with_pi=False)
    gF = op.filter(sino.astype(np.float64), v0, v1 - v0 + 1)
    want = oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb))
    got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    assert rel_l2(got, want) < TOL
    assert np.isfinite(vol).all()
    assert kp.info["update_count"] > 4.0e10
    import paper_2201_02309_b300 as kats
    assert kats.native.katsevich_device_status(kp.handle) == 0


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_c2_host_pipeline_matches_device(c2, prec):
    """katsevich_recon_host at full size (8 overlapped window chunks, 4 volume
    slabs) gives bit for bit the device-buffer result of katsevich_recon."""
    import torch

    import paper_2201_02309_b300 as kats
    g, sino, kp, dsino, vol = c2
    p = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16}[prec]
    dev = vol if prec == "fp32" else kp.recon(dsino, precision=p).cpu().numpy()
    hs = torch.from_numpy(sino).pin_memory()
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(hs, hv, precision=p)
    assert np.array_equal(hv.numpy(), dev)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_host_pipeline_small_volume_long_window(prec):
    """The overlapped host path on a 64 x 64 x 48 volume of the clinical scanner:
    its view window (about 1300 views of 64 x 736, above the pipeline's 128 MiB
    threshold) arrives in chunks, the first 16-slice slab is backprojected chunk
    by chunk from raw partial sums, and the result equals the device-buffer
    reconstruction bit for bit."""
    import torch

    import paper_2201_02309_b300 as kats
    cfg = dict(synth.config(2))
    cfg.update(nx=64, ny=64, nz=48)
    g = kats.make_geometry(cfg)
    kp = kats.Plan(g)
    nf = kp.info["n_filtered_views"]
    assert (nf + 1) * g["n_rows"] * g["n_cols"] * 4 >= (128 << 20)
    p = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16, "bf16": kats.KATS_PREC_BF16}[prec]
    rng = np.random.default_rng(5)
    sino = rng.standard_normal(kp.sino_shape).astype(np.float32)
    dev = kp.recon(torch.from_numpy(sino).cuda(), precision=p).cpu().numpy()
    hs = torch.from_numpy(sino).pin_memory()
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(hs, hv, precision=p)
    assert np.array_equal(hv.numpy(), dev)
    assert np.isfinite(dev).all() and np.abs(dev).max() > 0
