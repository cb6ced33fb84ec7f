"""Whole-operator pins of the oracle: reconstruction of analytic phantoms,
linearity, and a brute-force check that the adjoint is the exact transpose."""
import numpy as np
import pytest
from scipy.ndimage import binary_erosion

import oracle
import synth


@pytest.fixture(scope="module")
def c1():
    cfg = synth.config(1)
    g = oracle.derive_geometry(cfg)
    return cfg, g, oracle.Plan(g)


def voxel_centres(g):
    xs = g["x0"] + np.arange(g["nx"]) * g["dx"]
    ys = g["y0"] + np.arange(g["ny"]) * g["dy"]
    zs = g["z_first"] + np.arange(g["nz"]) * g["dz"]
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X, Y, Z], -1)


def test_uniform_ball(c1):
    # Katsevich's formula is exact: a uniform ball comes back at its density.
    _, g, pl = c1
    zc = g["z_first"] + 0.5 * (g["nz"] - 1) * g["dz"]
    sino = synth.project(g, synth.ball((0.0, 0.0, zc), 20.0))
    vol = pl.recon(sino)
    P = voxel_centres(g)
    r = np.linalg.norm(P - np.array([0, 0, zc]), axis=-1)
    inside, outside = r < 17.0, (r > 23.0) & (np.hypot(P[..., 0], P[..., 1]) < 30)
    assert abs(vol[inside].mean() - 1.0) < 2e-3
    assert np.abs(vol[inside] - 1.0).max() < 1e-2
    assert np.abs(vol[outside]).mean() < 1.2e-2
    assert np.abs(vol[outside]).max() < 6e-2


def test_off_centre_ball_and_hard_endpoints(c1):
    # An off-axis, off-centre ball pins the orientation conventions (a mirrored
    # alpha or a reversed view order would misplace or smear it).
    _, g, pl = c1
    zc = g["z_first"] + 0.5 * (g["nz"] - 1) * g["dz"] + 4.0
    ctr = np.array([12.0, -8.0, zc])
    sino = synth.project(g, synth.ball(ctr, 8.0))
    P = voxel_centres(g)
    r = np.linalg.norm(P - ctr, axis=-1)
    for mode, tol in ((0, 4e-3), (1, 1e-2)):
        gg = dict(g)
        gg["endpoint_mode"] = mode
        vol = oracle.Plan(gg).recon(sino) if mode else pl.recon(sino)
        assert abs(vol[r < 5.5].mean() - 1.0) < tol
        out = np.abs(vol[(r > 11) & (np.hypot(P[..., 0], P[..., 1]) < 30)])
        assert out.mean() < 1.2e-2 and out.max() < 6e-2


def test_shepp_style_levels(c1):
    cfg, g, pl = c1
    ell = synth.phantom_for(cfg, g, synth.phantom_seed(1))
    sino = synth.add_noise(synth.project(g, ell), cfg["noise_sigma"], synth.noise_seed(1))
    vol = pl.recon(sino)
    truth = synth.density(ell, voxel_centres(g).reshape(-1, 3)).reshape(vol.shape)
    checked = 0
    for v in np.unique(np.round(truth, 9)):
        m = binary_erosion(np.isclose(truth, v, atol=1e-9), iterations=2)
        if m.sum() < 30:
            continue
        checked += 1
        assert abs(vol[m].mean() - v) < 5e-3, v
    assert checked >= 3


def test_linearity(c1):
    _, g, pl = c1
    rng = np.random.default_rng(4)
    a = rng.normal(size=(g["n_views"], g["n_rows"], g["n_cols"]))
    b = rng.normal(size=a.shape)
    lhs = pl.recon(2.5 * a - 0.75 * b)
    rhs = 2.5 * pl.recon(a) - 0.75 * pl.recon(b)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))


def tiny_geometry(endpoint_mode=0):
    cfg = dict(R=20.0, D=40.0, views_per_turn=24, turns=3, n_rows=4, n_cols=8, n_cols_full=8, col_keep=1,
               det_half_width=4.0, nx=8, ny=8, nz=4, voxel=1.0, pitch_factor=1.0, endpoint_mode=endpoint_mode)
    return oracle.derive_geometry(cfg)


@pytest.mark.parametrize("mode", [0, 1])
def test_adjoint_is_dense_transpose(mode):
    # Build the operator matrix column by column and its adjoint row by row.
    g = tiny_geometry(mode)
    pl = oracle.Plan(g)
    n_in = g["n_views"] * g["n_rows"] * g["n_cols"]
    n_out = g["nx"] * g["ny"] * g["nz"]
    A = np.empty((n_out, n_in))
    e = np.zeros(n_in)
    for i in range(n_in):
        e[i] = 1.0
        A[:, i] = pl.recon(e.reshape(g["n_views"], g["n_rows"], g["n_cols"])).reshape(-1)
        e[i] = 0.0
    At = np.empty((n_in, n_out))
    u = np.zeros(n_out)
    for j in range(n_out):
        u[j] = 1.0
        At[:, j] = pl.adjoint(u.reshape(g["nz"], g["ny"], g["nx"])).reshape(-1)
        u[j] = 0.0
    assert np.abs(A).max() > 0
    assert np.max(np.abs(At - A.T)) <= 1e-12 * np.abs(A).max()


def test_adjoint_dot_product_c1(c1):
    _, g, pl = c1
    rng = np.random.default_rng(6)
    x = rng.normal(size=(g["n_views"], g["n_rows"], g["n_cols"]))
    y = rng.normal(size=(g["nz"], g["ny"], g["nx"]))
    lhs = float(np.sum(pl.recon(x) * y))
    rhs = float(np.sum(x * pl.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_table_periodicity(c1):
    # One-pitch tables serve every pitch: shifting the volume by one pitch
    # shifts every view index by one turn (Sec. II periodic properties).
    _, g, pl = c1
    g2 = dict(g)
    g2["z_first"] = g["z_first"] + g["P"]
    t2 = oracle.pi_table(g2)
    t1 = pl.pi
    assert np.array_equal(t2["k0"], t1["k0"] + g["views_per_turn"])
    assert np.array_equal(t2["k1"], t1["k1"] + g["views_per_turn"])
    assert np.allclose(t2["w0"], t1["w0"], atol=1e-9) and np.allclose(t2["w1"], t1["w1"], atol=1e-9)
    # end weights lie in (0, 1] and windows are sensible
    assert (t1["w0"] > 0).all() and (t1["w0"] <= 1).all() and (t1["w1"] > 0).all() and (t1["w1"] <= 1).all()


def test_point_windows_match_table(c1):
    _, g, pl = c1
    rng = np.random.default_rng(8)
    ijk = np.stack([rng.integers(0, g["nx"], 50), rng.integers(0, g["ny"], 50), rng.integers(0, g["nz"], 50)], 1)
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    N = oracle.pitch_slices(g)
    for p, (i, j, s) in enumerate(ijk):
        jj, m = s % N, s // N
        assert ka[p] == pl.pi["k0"][jj, j, i] + m * g["views_per_turn"]
        assert kb[p] == pl.pi["k1"][jj, j, i] + m * g["views_per_turn"]
    gF = pl.filter(synth.random_sino((g["n_views"], g["n_rows"], g["n_cols"]), 3))
    vol = pl.backproject(gF)
    pts = oracle.backproject_points(g, gF, 0, ijk)
    assert np.allclose(pts, vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]], rtol=1e-13, atol=1e-13)


def test_ellipsoid_line_integrals_vs_quadrature():
    # Input generator pin: closed-form chord vs 1-D quadrature of the indicator.
    rng = np.random.default_rng(12)
    q = rng.normal(size=4)
    ell = np.stack([synth.ellipsoid((3.0, -2.0, 5.0), (10.0, 6.0, 14.0), 0.7, synth._rotation(q))])
    src = np.array([[-60.0, 0.0, 0.0]] * 40) + rng.normal(scale=3.0, size=(40, 3))
    tgt = np.array([3.0, -2.0, 5.0]) + rng.normal(scale=5.0, size=(40, 3))
    d = tgt - src
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = synth.project_rays(ell, src, d)
    t = np.linspace(0, 130, 260001)
    for k in range(40):
        pts = src[k][None] + t[:, None] * d[k][None]
        ref = synth.density(ell, pts).sum() * (t[1] - t[0])
        assert abs(got[k] - ref) < 2 * 0.7 * (t[1] - t[0]) + 1e-12
    assert (got > 0).sum() > 20
