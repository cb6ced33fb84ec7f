"""Precision form: derivative and filtered data stored in BF16 / FP16, Hilbert on
16-bit tensor cores with a hi + lo Toeplitz operand, FP32 accumulation.
Bar: rel-L2 <= 1e-3 against the FP64 oracle; max-abs error reported."""
import numpy as np
import pytest

import oracle
import synth
from cases import c1_case, max_abs_rel, rel_l2

pytestmark = pytest.mark.gpu
TOL16 = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as kats
    return torch, kats


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_c1_reduced_precision(env, prec):
    torch, kats = env
    p = {"bf16": kats.KATS_PREC_BF16, "fp16": kats.KATS_PREC_FP16}[prec]
    _, g, sino = c1_case()
    kp = kats.Plan(g)
    vol = kp.recon(torch.from_numpy(sino).cuda(), precision=p).cpu().numpy()
    want = oracle.Plan(g).recon(sino.astype(np.float64))
    err = rel_l2(vol, want)
    print(f"{prec}: rel-L2 {err:.2e}, max-abs {np.abs(vol - want).max():.2e} (|f| max {np.abs(want).max():.2f})")
    assert err < TOL16


@pytest.fixture(scope="module")
def c4():
    """The mixed-precision workload at its stated size: the clinical geometry (512 x 512 x 256,
    64 x 736 detector, 8 turns) with a random-ellipsoid phantom's analytic projections."""
    cfg = synth.config(4)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(cfg, g, synth.phantom_seed(4))
    return g, synth.project(g, ell).astype(np.float32)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_c2_reduced_precision_sampled(env, c4, prec):
    torch, kats = env
    p = {"bf16": kats.KATS_PREC_BF16, "fp16": kats.KATS_PREC_FP16}[prec]
    g, sino = c4
    kp = kats.Plan(g)
    vol = kp.recon(torch.from_numpy(sino).cuda(), precision=p).cpu().numpy()
    rng = np.random.default_rng(4)
    n = 160
    ijk = np.stack([rng.integers(0, 512, n), rng.integers(0, 512, n), rng.integers(60, 62, n)], 1)
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    v0 = int(ka.min())
    gF = oracle.Plan(g, with_pi=False).filter(sino.astype(np.float64), v0, int(kb.max()) - v0 + 1)
    want = oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb))
    got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    err = rel_l2(got, want)
    print(f"{prec} full size: rel-L2 {err:.2e}, max-abs {np.abs(got - want).max():.2e}")
    assert err < TOL16
    assert np.isfinite(vol).all()


def test_reduced_precision_limits(env):
    torch, kats = env
    _, g, sino = c1_case()
    kp = kats.Plan(g)
    with pytest.raises(kats.KatsevichError) as e:
        kp.adjoint(torch.zeros(kp.vol_shape, device="cuda"), precision=kats.KATS_PREC_BF16)
    assert e.value.status == kats.native.KATS_EINVAL


def test_c4_reduced_precision_boundary_slices(env, c4):
    """Both 16-bit forms on the voxels where their launches change: the first and last 16-slice
    tiles, both sides of the pitch boundaries (69/70/71, 139/140, where the slice groups one pitch
    apart begin and end), the corner columns (the longest ramps) and a 16 x 16 tile boundary,
    against the oracle's chain on exactly the views each group of slices needs: rel-L2 <= 1e-3 per
    group, max-abs printed."""
    torch, kats = env
    g, sino = c4
    kp = kats.Plan(g)
    dsino = torch.from_numpy(sino).cuda()
    vols = {prec: kp.recon(dsino, precision=p).cpu().numpy()
            for prec, p in (("bf16", kats.KATS_PREC_BF16), ("fp16", kats.KATS_PREC_FP16))}
    del dsino
    op = oracle.Plan(g, with_pi=False)
    rng = np.random.default_rng(14)
    cols = [(0, 0), (511, 0), (0, 511), (511, 511), (15, 15), (16, 16), (15, 16), (16, 15), (255, 256)]
    for group in ([0, 15, 16], [69, 70, 71], [139, 140], [255]):
        ijk = []
        for s in group:
            ijk += [(i, j, s) for i, j in cols]
            ijk += [(int(i), int(j), s) for i, j in rng.integers(64, 448, (30, 2))]
        ijk = np.array(ijk)
        ka, kb, wa, wb = oracle.pi_windows(g, ijk)
        v0, v1 = int(ka.min()), int(kb.max())
        gF = op.filter(sino.astype(np.float64), v0, v1 - v0 + 1)
        want = oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb))
        for prec, vol in vols.items():
            got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
            err = rel_l2(got, want)
            print(f"{prec} slices {group}: rel-L2 {err:.2e}, max-abs / max {max_abs_rel(got, want):.2e}")
            assert err < TOL16 and np.isfinite(got).all()
