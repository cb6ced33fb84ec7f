"""GPU path vs the FP64 oracle, through the C ABI (via the ctypes binding).

Bars: integer tables bit-exact (a mismatch is allowed only where the oracle's
fractional part is within 1e-9 of an integer, i.e. a floor tie between two
correctly rounded FP64 evaluations); FP32 results within rel-L2 1e-5 of the
oracle on the same FP32-rounded input.
"""
import numpy as np
import pytest

import oracle
from cases import c1_case, check32, finevoxel_case, fourpitch_case, multipitch_case, narrow_case, near_tie, odd_case, rel_l2, rows80_case, tall_case

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def kats():
    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as k
    return k


def check_int_table(got, want, want_frac, name):
    bad = got != want
    if bad.any():
        ties = near_tie(want_frac)
        assert not (bad & ~ties).any(), f"{name}: {int((bad & ~ties).sum())} mismatches away from ties"
    return int(bad.sum())


def compare_tables(kp, op):
    assert check_int_table(kp.table("kappa_idx"), op.kap[0], op.kap[1], "kappa") <= 2
    same = kp.table("kappa_idx") == op.kap[0]
    assert np.abs(kp.table("kappa_frac") - op.kap[1])[same].max() < 2e-7
    assert check_int_table(kp.table("psi_idx"), op.psi[0], op.psi[1], "psi") <= 2
    same = kp.table("psi_idx") == op.psi[0]
    assert np.abs(kp.table("psi_frac") - op.psi[1])[same].max() < 2e-7
    if op.pi is not None:
        for a, b in (("k0", "w0"), ("k1", "w1")):
            n = check_int_table(kp.table(a), op.pi[a], op.pi[b], a)
            assert n <= 2
            same = kp.table(a) == op.pi[a]
            assert np.abs(kp.table(b) - op.pi[b])[same].max() < 2e-7


@pytest.fixture(scope="module")
def c1(kats):
    cfg, g, sino = c1_case()
    return g, sino, oracle.Plan(g), kats.Plan(g)


def test_tables_c1(c1):
    g, _, op, kp = c1
    compare_tables(kp, op)


def test_plan_info_c1(c1):
    g, _, op, kp = c1
    info = kp.info
    N = oracle.pitch_slices(g)
    assert info["slices_per_pitch"] == N
    assert info["update_count"] == op.update_count()
    s = np.arange(g["nz"])
    kmin = min(int(op.pi["k0"][j].min()) + (ss // N) * g["views_per_turn"] for ss, j in zip(s, s % N))
    kmax = max(int(op.pi["k1"][j].max()) + (ss // N) * g["views_per_turn"] for ss, j in zip(s, s % N))
    assert info["first_view"] == kmin and info["n_filtered_views"] == kmax - kmin + 1
    ext = op.extents()
    assert abs(info["lambda_min"] - ext[0]) < 1e-12 and abs(info["lambda_max"] - ext[1]) < 1e-12
    assert np.allclose([info["alpha_min"], info["alpha_max"]], ext[2:4], rtol=1e-5, atol=1e-7)
    assert np.allclose([info["w_min"], info["w_max"]], ext[4:6], rtol=1e-5, atol=1e-5)
    assert info["alpha_m"] == pytest.approx(oracle.alpha_m(g), rel=1e-15)
    # window starts / ends nondecreasing slice to slice (FP32 end weights as stored)
    t = op.pi
    s0 = t["k0"] - t["w0"].astype(np.float32).astype(np.float64)
    e0 = t["k1"] + t["w1"].astype(np.float32).astype(np.float64)
    s0 = np.concatenate([s0, s0[:1] + g["views_per_turn"]], 0)
    e0 = np.concatenate([e0, e0[:1] + g["views_per_turn"]], 0)
    mono = bool(np.all(np.diff(s0, axis=0) >= 0) and np.all(np.diff(e0, axis=0) >= 0))
    assert mono and info["pi_monotone"] == 1


def test_pi_endpoints_fp64(kats):
    _, g, _ = odd_case()
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(-0.9, 0.9, 400) * 200, rng.uniform(-0.9, 0.9, 400) * 200,
                    rng.uniform(-300, 300, 400)], 1)
    pts[0] = (0.0, 0.0, 12.5)
    li, lo = kats.pi_endpoints(g, pts)
    want = np.array([oracle.pi_endpoints(g, *p) for p in pts])
    assert np.abs(li - want[:, 0]).max() < 1e-11
    assert np.abs(lo - want[:, 1]).max() < 1e-11


def pad_cols(gF, gcols):
    out = np.zeros(gF.shape[:-1] + (gcols,), np.float32)
    out[..., :gF.shape[-1]] = gF
    return out


def test_filter_parity_c1(c1, torch):
    g, sino, op, kp = c1
    gF = kp.filter(torch.from_numpy(sino).cuda()).cpu().numpy()
    v0, nv = kp.info["first_view"], kp.info["n_filtered_views"]
    want = op.filter(sino.astype(np.float64), v0, nv)
    assert gF.shape[-1] == kp.info["gf_cols"] and kp.info["gf_cols"] % 4 == 0
    assert not gF[..., g["n_cols"]:].any()
    check32(gF[..., :g["n_cols"]], want)


def test_backproject_parity_c1(c1, torch):
    g, sino, op, kp = c1
    v0, nv = kp.info["first_view"], kp.info["n_filtered_views"]
    gF = op.filter(sino.astype(np.float64), v0, nv).astype(np.float32)
    vol = kp.backproject(torch.from_numpy(pad_cols(gF, kp.info["gf_cols"])).cuda()).cpu().numpy()
    want = op.backproject(gF.astype(np.float64), v0)
    check32(vol, want)


def test_recon_parity_c1(c1, torch):
    g, sino, op, kp = c1
    vol = kp.recon(torch.from_numpy(sino).cuda()).cpu().numpy()
    want = op.recon(sino.astype(np.float64))
    check32(vol, want)


def test_adjoint_parity_c1(c1, torch):
    g, _, op, kp = c1
    rng = np.random.default_rng(9)
    y = rng.normal(size=kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    want = op.adjoint(y.astype(np.float64))
    check32(got, want)


@pytest.mark.parametrize("mode", [0, 1])
def test_multipitch_ragged(kats, torch, mode):
    _, g, sino = multipitch_case(mode)
    op, kp = oracle.Plan(g), kats.Plan(g)
    compare_tables(kp, op)
    assert kp.info["update_count"] == op.update_count()
    vol = kp.recon(torch.from_numpy(sino).cuda()).cpu().numpy()
    check32(vol, op.recon(sino.astype(np.float64)))
    y = np.random.default_rng(1).normal(size=kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    check32(got, op.adjoint(y.astype(np.float64)))


def test_fourpitch_bands(kats, torch):
    """Four and three slice groups one pitch apart per thread, each view staged as a band of rows
    (fp32 against the oracle at the FP32 bar, the 16-bit forms at theirs), and the same volume
    from slab launches that group the slices differently."""
    _, g, sino = fourpitch_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    want = op.recon(sino.astype(np.float64))
    dsino = torch.from_numpy(sino).cuda()
    vol = kp.recon(dsino).cpu().numpy()
    check32(vol, want)
    for p in (kats.KATS_PREC_FP16, kats.KATS_PREC_BF16):
        assert rel_l2(kp.recon(dsino, precision=p).cpu().numpy(), want) < 1e-3
    # slices [48, 194): leading slices 48-77 take three groups and 78-105 two, a different grouping
    slab = kp.recon_slab(dsino.clone(), 0, 48, 194).cpu().numpy()
    check32(slab, want[48:], name="slab 48-194")


def test_fine_voxel_bands(kats, torch):
    """Slice groups and row bands on 0.8 mm voxels (the band bound scales with dz and the voxel
    spacing): FP32 against the oracle, and the 16-bit forms at their bar."""
    _, g, sino = finevoxel_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    assert kp.info["slices_per_pitch"] == 60
    want = op.recon(sino.astype(np.float64))
    dsino = torch.from_numpy(sino).cuda()
    check32(kp.recon(dsino).cpu().numpy(), want)
    for p in (kats.KATS_PREC_FP16, kats.KATS_PREC_BF16):
        assert rel_l2(kp.recon(dsino, precision=p).cpu().numpy(), want) < 1e-3


def test_odd_offsets_slice_groups(kats, torch):
    """Every offset of the odd geometry (lambda0, z0, lambda_first, alpha and w) with a volume of
    three pitches: four- and three-group items, row bands."""
    _, g, sino = odd_case(tall=True)
    op, kp = oracle.Plan(g), kats.Plan(g)
    compare_tables(kp, op)
    want = op.recon(sino.astype(np.float64))
    dsino = torch.from_numpy(sino).cuda()
    check32(kp.recon(dsino).cpu().numpy(), want)
    assert rel_l2(kp.recon(dsino, precision=kats.KATS_PREC_FP16).cpu().numpy(), want) < 1e-3


def test_odd_geometry_batch(kats, torch):
    _, g, sino = odd_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    compare_tables(kp, op)
    batch = np.stack([sino, -0.5 * sino + 0.1])
    vol = kp.recon(torch.from_numpy(batch).cuda()).cpu().numpy()
    for b in range(2):
        check32(vol[b], op.recon(batch[b].astype(np.float64)))
    y = np.random.default_rng(3).normal(size=(2,) + kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    for b in range(2):
        check32(got[b], op.adjoint(y[b].astype(np.float64)))


def test_four_slot_ring(kats, torch):
    """80 detector rows: the staged backprojection runs its ring with two slot pairs."""
    _, g, sino = rows80_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    want = op.recon(sino.astype(np.float64))
    dsino = torch.from_numpy(sino).cuda()
    check32(kp.recon(dsino).cpu().numpy(), want)
    for p in (kats.KATS_PREC_FP16, kats.KATS_PREC_BF16):
        assert rel_l2(kp.recon(dsino, precision=p).cpu().numpy(), want) < 1e-3
    # the host-buffer path gives the same volume bit for bit
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(torch.from_numpy(sino).pin_memory(), hv)
    assert np.array_equal(hv.numpy(), kp.recon(dsino).cpu().numpy())


def test_tall_detector_uncached_tables(kats, torch):
    _, g, sino = tall_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    assert kp.info["n_psi"] == 528
    compare_tables(kp, op)
    vol = kp.recon(torch.from_numpy(sino).cuda()).cpu().numpy()
    check32(vol, op.recon(sino.astype(np.float64)))
    y = np.random.default_rng(2).normal(size=kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    check32(got, op.adjoint(y.astype(np.float64)))
    # the reduced-precision backprojection needs the staged window: refused, not wrong
    with pytest.raises(kats.KatsevichError) as e:
        kp.recon(torch.from_numpy(sino).cuda(), precision=kats.KATS_PREC_FP16)
    assert e.value.status == kats.native.KATS_EINVAL


def test_narrow_detector_fallback_path(kats, torch):
    # 9-column detector: too narrow for the staged window, so the global-memory kernel runs
    _, g, sino = narrow_case()
    op, kp = oracle.Plan(g), kats.Plan(g)
    compare_tables(kp, op)
    vol = kp.recon(torch.from_numpy(sino).cuda()).cpu().numpy()
    check32(vol, op.recon(sino.astype(np.float64)))
    y = np.random.default_rng(2).normal(size=kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    check32(got, op.adjoint(y.astype(np.float64)))


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 17, 3), (33, 1, 1), (17, 18, 1)])
def test_degenerate_volumes(kats, torch, shape):
    """Volumes one voxel wide, high or deep: partly empty 16 x 16 x 16 tiles, single slices, a
    single voxel column; recon and adjoint against the oracle, host path bit for bit."""
    import synth
    cfg = dict(synth.config(1))
    cfg.update(nx=shape[0], ny=shape[1], nz=shape[2])
    g = oracle.derive_geometry(cfg)
    sino = np.random.default_rng(sum(shape)).normal(size=(g["n_views"], g["n_rows"], g["n_cols"])).astype(np.float32)
    op, kp = oracle.Plan(g), kats.Plan(g)
    assert kp.info["update_count"] == op.update_count()
    dsino = torch.from_numpy(sino).cuda()
    vol = kp.recon(dsino).cpu().numpy()
    assert vol.shape == (shape[2], shape[1], shape[0])
    check32(vol, op.recon(sino.astype(np.float64)))
    y = np.random.default_rng(1).normal(size=kp.vol_shape).astype(np.float32)
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    check32(got, op.adjoint(y.astype(np.float64)))
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(torch.from_numpy(sino).pin_memory(), hv)
    assert np.array_equal(hv.numpy(), vol)


def test_device_status_clean(c1, kats):
    _, _, _, kp = c1
    assert kats.native.katsevich_device_status(kp.handle) == 0


def test_recon_host_matches_device(c1, torch):
    g, sino, op, kp = c1
    dev = kp.recon(torch.from_numpy(sino).cuda()).cpu()
    hs = torch.from_numpy(sino).pin_memory()
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(hs, hv)
    assert torch.equal(dev, hv)


def test_errors(c1, torch, kats):
    g, sino, op, kp = c1
    x = torch.from_numpy(sino).cuda()
    out = torch.empty(kp.vol_shape, device="cuda")
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(kats.KatsevichError) as e:
        kp.recon(x, out=out, workspace=small)
    assert e.value.status == kats.native.KATS_ESPACE
    with pytest.raises(kats.KatsevichError) as e:
        kats.native.katsevich_recon(kp.handle, x.data_ptr(), out.data_ptr(), 0, 0, small.data_ptr(), 16, 0)
    assert e.value.status == kats.native.KATS_EINVAL
    with pytest.raises(ValueError):
        kp.recon(x[:-1].contiguous())
    # a volume whose PI windows leave the scan is rejected at plan time
    g2 = dict(g)
    g2["z_first"] = g["z_first"] + 4 * g["P"]
    with pytest.raises(kats.KatsevichError) as e:
        kats.Plan(g2)
    assert e.value.status == kats.native.KATS_EGEOM
