"""z-slab partition of one volume, the multi-GPU split of a single reconstruction
(one slab per rank, no exchange between them): a slab computed from only the
sinogram views it reads equals those slices of the whole-volume reconstruction
(bit for bit where the slab and the whole volume group their slices alike, to FP32
rounding where the multi-pitch kernel groups a slice differently), and the views it
reads are the union of its voxels' PI windows, taken here from the plan's one-pitch
k0 / k1 tables shifted by whole turns."""
import numpy as np
import pytest

import synth
from cases import close_paths, multipitch_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kats():
    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as k
    return k


def expected_views(kp, s0, s1):
    """Sinogram views [begin, begin + count) that slices [s0, s1) read: half-views k0 .. k1 of
    every voxel's PI window, each formed from views k and k + 1."""
    k0, k1 = kp.table("k0").astype(np.int64), kp.table("k1").astype(np.int64)
    n, vpt = kp.info["slices_per_pitch"], kp.geom["views_per_turn"]
    lo, hi = None, None
    for s in range(s0, s1):
        a, b = k0[s % n], k1[s % n]
        ok = a <= b
        if not ok.any():
            continue
        shift = (s // n) * vpt
        lo = a[ok].min() + shift if lo is None else min(lo, a[ok].min() + shift)
        hi = b[ok].max() + shift if hi is None else max(hi, b[ok].max() + shift)
    return (int(lo), int(hi - lo + 2)) if lo is not None else None


def run_slabs(kats, kp, dsino, world, prec):
    out = np.full(kp.vol_shape, np.nan, np.float32)
    spans = []
    for s0, s1 in kats.slab_partition(kp.geom["nz"], world):
        if s0 == s1:
            continue
        vb, vc = kp.slab_views(s0, s1)
        assert (vb, vc) == expected_views(kp, s0, s1)
        window = dsino[vb:vb + vc].clone()  # the rank holds only its views
        out[s0:s1] = kp.recon_slab(window, vb, s0, s1, precision=prec).cpu().numpy()
        spans.append((vb, vb + vc))
    return out, spans


def test_multipitch_slabs_equal_whole_volume(kats):
    import torch
    _, g, sino = multipitch_case(0)  # 150 slices over 2.6 pitches: slabs cut across pitch boundaries
    kp = kats.Plan(g)
    dsino = torch.from_numpy(sino).cuda()
    full = kp.recon(dsino).cpu().numpy()
    for world in (1, 2, 3, 4):
        out, spans = run_slabs(kats, kp, dsino, world, kats.KATS_PREC_FP32)
        if world == 1:  # one slab is the whole volume: the same launch
            assert np.array_equal(out, full)
        else:
            close_paths(out, full, f"{world} slabs")
        # a rank reads far fewer views than the scan holds; neighbours share a halo of views
        if world > 1:
            assert all(b0 < a1 for (_, a1), (b0, _) in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) < g["n_views"]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_clinical_scanner_slabs(kats, prec):
    import torch
    cfg = dict(synth.config(2))
    cfg.update(nx=64, ny=64, nz=80)
    g = kats.make_geometry(cfg)
    kp = kats.Plan(g)
    p = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16, "bf16": kats.KATS_PREC_BF16}[prec]
    dsino = torch.from_numpy(np.random.default_rng(11).standard_normal(kp.sino_shape).astype(np.float32)).cuda()
    full = kp.recon(dsino, precision=p).cpu().numpy()
    out, _ = run_slabs(kats, kp, dsino, 2, p)
    assert np.array_equal(out, full)
    assert np.isfinite(full).all() and np.abs(full).max() > 0


def test_slab_errors(kats):
    import torch
    _, g, sino = multipitch_case(0)
    kp = kats.Plan(g)
    dsino = torch.from_numpy(sino).cuda()
    vb, vc = kp.slab_views(16, 48)
    with pytest.raises(kats.KatsevichError):  # start off the 16-slice tile grid
        kp.recon_slab(dsino[vb:vb + vc].clone(), vb, 8, 48)
    with pytest.raises(kats.KatsevichError):  # window one view short
        kp.recon_slab(dsino[vb:vb + vc - 1].clone(), vb, 16, 48)
    with pytest.raises(kats.KatsevichError):  # window starting one view late
        kp.recon_slab(dsino[vb + 1:vb + vc + 1].clone(), vb + 1, 16, 48)
    for s0, s1 in ((0, 0), (40, 20), (0, g["nz"] + 1), (-16, 16)):
        with pytest.raises(kats.KatsevichError):
            kp.slab_views(s0, s1)
    # a wider window than needed is fine
    w0 = max(vb - 3, 0)
    a = kp.recon_slab(dsino[w0:vb + vc + 5].clone(), w0, 16, 48).cpu().numpy()
    b = kp.recon_slab(dsino[vb:vb + vc].clone(), vb, 16, 48).cpu().numpy()
    assert np.array_equal(a, b)
    close_paths(a, kp.recon(dsino).cpu().numpy()[16:48], "slab 16:48")
