"""Pins of the data-simulation oracle (the paper's Sec. III-C data
generation): helical projection of a voxel volume, sparse-detector
upsampling, and the Gaussian+Poisson noise model with its counter-based
generator.  Each pin comes from outside the oracle: published known-answer
vectors, closed-form ray/box intersection lengths computed here in numpy,
analytic line integrals of a ball from the input generator, exact linear
reproduction, and distribution tests against scipy's Poisson and normal
laws."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def small_geom(**kw):
    cfg = dict(synth.config(1))
    cfg.update(dict(dict(nx=24, ny=20, nz=12), **kw))
    return oracle.derive_geometry(cfg)


def slab_length(a, d, lo, hi):
    """Length of the line a + t d inside the box [lo, hi] (slab method)."""
    t0, t1 = -np.inf, np.inf
    for ax in range(3):
        if d[ax] == 0.0:
            if not (lo[ax] <= a[ax] <= hi[ax]):
                return 0.0
            continue
        ta, tb = (lo[ax] - a[ax]) / d[ax], (hi[ax] - a[ax]) / d[ax]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def box(g):
    lo = np.array([g["x0"] - 0.5 * g["dx"], g["y0"] - 0.5 * g["dy"], g["z_first"] - 0.5 * g["dz"]])
    hi = lo + np.array([g["nx"] * g["dx"], g["ny"] * g["dy"], g["nz"] * g["dz"]])
    return lo, hi


def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_rays_follow_acquisition_geometry():
    g = small_geom()
    dl = 2 * math.pi / g["views_per_turn"]
    for k, r, c in [(0, 0, 0), (17, 5, 100), (200, 31, 127), (383, 16, 64)]:
        a, d = oracle.ray(g, k, r, c)
        alpha = (c - 0.5 * (g["n_cols"] - 1)) * g["d_alpha"] + g["alpha_offset"]
        w = (r - 0.5 * (g["n_rows"] - 1)) * g["d_w"] + g["w_offset"]
        s, u = synth.ray(g, g["lambda_first"] + k * dl, alpha, w)
        assert np.allclose(a, s, atol=1e-9)
        assert np.allclose(d / np.linalg.norm(d), u, atol=1e-12)
        assert abs(np.linalg.norm(d) - math.hypot(g["D"], w)) < 1e-9  # a + d is the detector sample


def test_single_voxel_intersection_lengths():
    g = small_geom()
    rng = np.random.default_rng(3)
    lo, hi = box(g)
    checked = 0
    mid = g["n_views"] // 2  # views whose rays cross the (thin) volume
    for k in rng.integers(mid - 30, mid + 30, 10):
        rows = rng.integers(g["n_rows"] // 2 - 8, g["n_rows"] // 2 + 8, 12)
        cols = rng.integers(g["n_cols"] // 2 - 15, g["n_cols"] // 2 + 15, 12)  # the narrow volume's shadow
        for r, c in zip(rows, cols):
            a, d = oracle.ray(g, int(k), int(r), int(c))
            L = slab_length(a, d, lo, hi)
            if L == 0.0:
                continue
            # a voxel the ray crosses: the one holding a random point of the chord
            t0 = max(min((lo[i] - a[i]) / d[i], (hi[i] - a[i]) / d[i]) for i in range(3) if d[i] != 0)
            p = a + (t0 + rng.uniform(0.2, 0.8) * L / np.linalg.norm(d)) * d
            idx = np.floor((p - (lo)) / np.array([g["dx"], g["dy"], g["dz"]])).astype(int)
            vol = np.zeros((g["nz"], g["ny"], g["nx"]))
            vol[idx[2], idx[1], idx[0]] = 1.0
            got = oracle.project(g, vol, int(k), 1)[0, r, c]
            vlo = lo + idx * np.array([g["dx"], g["dy"], g["dz"]])
            want = slab_length(a, d, vlo, vlo + np.array([g["dx"], g["dy"], g["dz"]]))
            assert abs(got - want) < 1e-9, (k, r, c, idx, got, want)
            checked += 1
    assert checked > 20


def test_constant_volume_gives_chord_lengths():
    g = small_geom()
    lo, hi = box(g)
    v0 = g["n_views"] // 2 - 1
    got = oracle.project(g, np.ones((g["nz"], g["ny"], g["nx"])), v0, 2)
    assert got.max() > 10.0
    for v in range(2):
        for r in range(0, g["n_rows"], 5):
            for c in range(0, g["n_cols"], 9):
                a, d = oracle.ray(g, v0 + v, r, c)
                assert abs(got[v, r, c] - slab_length(a, d, lo, hi)) < 1e-9


def ball_projection_error(vox):
    """rel-L2 and total-mass ratio of the projection of a voxelized ball (4^3
    sub-sample voxel averages) against its analytic line integrals."""
    n = int(round(40 / vox))
    g = small_geom(nx=n, ny=n, nz=int(round(24 / vox)), voxel=vox)
    zc = g["z_first"] + 0.5 * (g["nz"] - 1) * g["dz"]
    ball = synth.ball((2.0, -1.5, zc), 9.0)
    sub = (np.arange(4) + 0.5) / 4 - 0.5
    xs = g["x0"] + np.add.outer(np.arange(g["nx"]), sub).ravel() * g["dx"]
    ys = g["y0"] + np.add.outer(np.arange(g["ny"]), sub).ravel() * g["dy"]
    zs = g["z_first"] + np.add.outer(np.arange(g["nz"]), sub).ravel() * g["dz"]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    dens = synth.density(ball, np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)).reshape(Z.shape)
    vol = dens.reshape(g["nz"], 4, g["ny"], 4, g["nx"], 4).mean(axis=(1, 3, 5))
    views = [g["n_views"] // 2 + o for o in (-20, 0, 35)]
    got = np.stack([oracle.project(g, vol, v, 1)[0] for v in views])
    want = np.stack([synth.project(g, ball, v, 1)[0] for v in views])
    return np.linalg.norm(got - want) / np.linalg.norm(want), got.sum() / want.sum(), got.max() / want.max()


def test_voxelized_ball_converges_to_analytic_integrals():
    """Same geometry conventions as the analytic projector: the error is the
    voxelization of the ball's edge, first order in the voxel size."""
    e1, m1, p1 = ball_projection_error(1.0)
    e2, m2, p2 = ball_projection_error(0.5)
    assert e1 < 0.08 and e2 < 0.6 * e1, (e1, e2)
    assert abs(m1 - 1) < 1e-2 and abs(m2 - 1) < 1e-2 and abs(p1 - 1) < 1e-2 and abs(p2 - 1) < 1e-2


def test_projection_is_linear():
    g = small_geom()
    rng = np.random.default_rng(1)
    f1, f2 = rng.normal(size=(2, g["nz"], g["ny"], g["nx"]))
    p = lambda f: oracle.project(g, f, g["n_views"] // 2, 2)
    assert np.allclose(p(2 * f1 - 0.5 * f2), 2 * p(f1) - 0.5 * p(f2), atol=1e-10)


def test_sparse_upsample_reproduces_kept_columns_and_lines():
    g = small_geom()
    nc, keep = g["n_cols"], 4
    c = np.arange(nc, dtype=np.float64)
    last = (nc - 1) // keep * keep
    sino = np.empty((3, g["n_rows"], nc))
    sino[:] = 0.7 * c - 3.0  # linear along the columns
    out = oracle.sparse_upsample(g, sino, keep)
    assert np.allclose(out[..., : last + 1], sino[..., : last + 1], atol=1e-12)
    assert np.all(out[..., last:] == sino[..., last:last + 1])  # beyond the last kept column: its value
    rnd = np.random.default_rng(2).normal(size=sino.shape)
    out = oracle.sparse_upsample(g, rnd, keep)
    assert np.array_equal(out[..., ::keep], rnd[..., ::keep])


@pytest.mark.parametrize("lam", [3.7, 50.0, 1.0e5])
def test_poisson_draws_follow_the_poisson_law(lam):
    n = 20000
    k = np.array([oracle.poisson(lam, 12345, i) for i in range(n)])
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / n)
    assert abs(k.var() / lam - 1) < 5 * math.sqrt(2.0 / n)
    # chi-square against the exact pmf over bins holding >= 20 expected draws
    lo, hi = stats.poisson.ppf([1e-4, 1 - 1e-4], lam).astype(int)
    edges = np.unique(np.linspace(lo, hi + 1, min(hi - lo + 2, 40)).astype(int))
    obs = np.histogram(k, bins=edges)[0]
    exp = n * np.diff(stats.poisson.cdf(edges - 1, lam))
    keep = exp >= 20
    chi2 = (((obs - exp) ** 2) / exp)[keep].sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_gaussian_draws_are_standard_normal():
    z = np.array([oracle.gaussian(777, i) for i in range(20000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # independent of the Poisson stream of the same samples
    k = np.array([oracle.poisson(1e5, 777, i) for i in range(20000)], dtype=np.float64)
    assert abs(np.corrcoef(z, k)[0, 1]) < 0.03


def test_noise_model_limits_and_moments():
    x = np.full(50000, 2.0)
    x[0] = 5.0  # M
    # no noise: I0 -> inf, var = 0 gives back the input (up to the Poisson relative spread 1/sqrt(I0))
    out, counts, M = oracle.add_noise(x, I0=1e14, mean=0.0, var=0.0, seed=1)
    assert M == 5.0 and np.abs(out - x).max() < 1e-5
    # moments at I0 = 1e5: counts ~ Poisson(I0 exp(-x/M)), g_in = M log(I0 / counts)
    out, counts, M = oracle.add_noise(x, I0=1e5, mean=0.0, var=0.5, seed=2)
    lam = 1e5 * math.exp(-2.0 / 5.0)
    c = counts[1:]
    assert abs(c.mean() - lam) < 5 * math.sqrt(lam / c.size)
    sd_expected = M * math.sqrt(1.0 / lam + 0.5 / lam ** 2)  # delta method
    assert abs(out[1:].mean() - 2.0) < 5 * sd_expected / math.sqrt(c.size) + M / (2 * lam)
    assert abs(out[1:].std() / sd_expected - 1) < 0.05
    # counts floor: with one photon most draws are 0 or 1; a zero count reads as one photon
    out, counts, M = oracle.add_noise(x, I0=1.0, mean=0.0, var=0.0, seed=3)
    assert np.isfinite(out).all() and (counts == 0).sum() > 1000
    assert np.all(out[counts == 0] == 0.0) and np.allclose(out[counts > 0], M * np.log(1.0 / counts[counts > 0]))
