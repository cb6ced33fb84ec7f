"""Data simulation on the GPU (the paper's Sec. III-C data generation) against
the FP64 oracle: helical projection (rel-L2 1e-5: FP32 traversal and
accumulation), sparse-detector upsampling (float rounding of one lerp), and
the Gaussian+Poisson noise (Poisson counts bit-exact: both sides draw from the
same counter-based generator with FP64 decisions; g_in within float
rounding)."""
import numpy as np
import pytest

import oracle
import synth
from cases import check32, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kats():
    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as k
    return k


def geom(**kw):
    cfg = dict(synth.config(1))
    cfg.update(dict(dict(nx=37, ny=29, nz=13), **kw))  # ragged sizes
    return oracle.derive_geometry(cfg)


def phantom_volume(g, seed=4):
    """Voxel-centre samples of the shepp-style phantom plus seeded texture."""
    zc = g["z_first"] + 0.5 * (g["nz"] - 1) * g["dz"]
    ell = synth.shepp_style(seed, 0.5 * min(g["nx"] * g["dx"], g["ny"] * g["dy"]), zc)
    z, y, x = np.meshgrid(g["z_first"] + g["dz"] * np.arange(g["nz"]), g["y0"] + g["dy"] * np.arange(g["ny"]),
                          g["x0"] + g["dx"] * np.arange(g["nx"]), indexing="ij")
    f = synth.density(ell, np.stack([x.ravel(), y.ravel(), z.ravel()], 1)).reshape(x.shape)
    return (f + 0.05 * np.random.default_rng(seed).random(f.shape)).astype(np.float32)


def test_projection_matches_oracle(kats):
    import torch
    g = geom()
    vol = phantom_volume(g)
    v0, nv = g["n_views"] // 2 - 40, 80
    got = kats.project(g, torch.from_numpy(vol).cuda(), v0, nv).cpu().numpy()
    want = oracle.project(g, vol.astype(np.float64), v0, nv)
    assert want.max() > 1.0
    check32(got, want)


def test_projection_clinical_views_match_oracle(kats):
    """Two views of the 512 x 512 x 256 clinical geometry (config 2).  Per element the bar is
    5e-5 x the largest ray sum: a ray crosses up to about 1500 voxel faces, and each face's
    FP32 ray parameter (t up to about 1700 mm, ulp 1.2e-4 mm) moves a segment's length by up
    to that much, so a random volume's ray sum carries about 1e-4 x sqrt(1500) mm of error."""
    import torch
    g = oracle.derive_geometry(synth.config(2))
    rng = np.random.default_rng(9)
    vol = rng.random((g["nz"], g["ny"], g["nx"]), dtype=np.float32)
    v = [g["n_views"] // 2, g["n_views"] // 2 + 577]
    dvol = torch.from_numpy(vol).cuda()
    for k in v:
        got = kats.project(g, dvol, k, 1).cpu().numpy()
        want = oracle.project(g, vol, k, 1)
        check32(got, want, elem_tol=5e-5)


def test_projection_of_every_view_is_finite_and_zero_outside(kats):
    import torch
    g = geom()
    vol = torch.ones((g["nz"], g["ny"], g["nx"]), device="cuda")
    sino = kats.project(g, vol).cpu().numpy()
    assert np.isfinite(sino).all() and sino.min() == 0.0 and sino.max() > 1.0
    want = oracle.project(g, np.ones((g["nz"], g["ny"], g["nx"])), 0, 3)  # views that miss the volume
    assert np.array_equal(sino[:3] == 0, want == 0)


def test_sparse_upsample_matches_oracle(kats):
    import torch
    g = geom()
    rng = np.random.default_rng(5)
    sino = rng.normal(size=(7, g["n_rows"], g["n_cols"])).astype(np.float32)
    for keep in (2, 4, 5):
        got = kats.sparse_upsample(g, torch.from_numpy(sino).cuda(), keep).cpu().numpy()
        want = oracle.sparse_upsample(g, sino, keep)
        assert np.abs(got - want).max() <= 4e-7 * np.abs(sino).max()
        assert np.array_equal(got[..., ::keep], sino[..., ::keep])


def test_noise_matches_oracle_draw_for_draw(kats):
    import torch
    g = geom()
    vol = phantom_volume(g)
    v0 = g["n_views"] // 2 - 20
    g_up = oracle.sparse_upsample(g, oracle.project(g, vol, v0, 40), 4).astype(np.float32)
    for I0, var, seed in [(1e5, 0.5, 11), (300.0, 2.0, 12), (5.0, 0.0, 13)]:
        got, M, counts = kats.add_noise(torch.from_numpy(g_up).cuda(), I0=I0, var=var, seed=seed,
                                        return_counts=True)
        want, want_counts, want_M = oracle.add_noise(g_up, I0=I0, mean=0.0, var=var, seed=seed)
        assert M == want_M == float(g_up.max())
        assert np.array_equal(counts.cpu().numpy(), want_counts), I0  # same generator, same draws
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-6 * max(1.0, np.abs(want).max())


def test_noise_draw_depends_only_on_index_and_seed(kats):
    import torch
    x = torch.linspace(0, 3, 100_000, device="cuda")
    x[0] = 4.0  # M in the prefix
    a, Ma, ca = kats.add_noise(x, seed=21, return_counts=True)
    b, Mb, cb = kats.add_noise(x[:5000].contiguous(), seed=21, return_counts=True)
    assert Ma == Mb and torch.equal(ca[:5000], cb) and torch.equal(a[:5000], b)
    c, _, cc = kats.add_noise(x, seed=22, return_counts=True)
    assert not torch.equal(ca, cc)


def test_simulated_input_reconstructs_the_label(kats):
    """Projection -> sparse upsampling -> noise -> reconstruction: the label
    comes back up to the sparse-detector and noise error."""
    import torch
    cfg = dict(synth.config(1))
    g = oracle.derive_geometry(cfg)
    vol = torch.from_numpy(phantom_volume(g)).cuda()
    g_gt, g_in = kats.simulate_input(g, vol, keep=2, I0=1e5, var=0.5, seed=3)
    plan = kats.Plan(g)
    rec_gt = plan.recon(g_gt)
    rec_in = plan.recon(g_in)
    inner = (slice(4, -4), slice(8, -8), slice(8, -8))
    e_gt = rel_l2(rec_gt[inner].cpu().numpy(), vol[inner].cpu().numpy())
    e_in = rel_l2(rec_in[inner].cpu().numpy(), vol[inner].cpu().numpy())
    assert e_gt < 0.3 and e_in < 0.45 and e_in > e_gt, (e_gt, e_in)  # FP64 oracle chain: 0.235, 0.348
