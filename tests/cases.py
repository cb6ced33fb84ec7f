"""Workload builders shared by the parity tests (geometry from the oracle's own
derivation, inputs from the seeded generator)."""
import math

import numpy as np

import oracle
import synth


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_abs_rel(a, b):
    """Largest element error relative to the largest expected magnitude."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def check32(got, want, tol=1e-5, name="", elem_tol=None):
    """The FP32 parity bar: rel-L2 <= tol over the array and, element by element,
    |got - want| <= elem_tol * max|want| (elem_tol = tol unless a test states its own), so that
    a wrong tile corner or slice cannot hide under the global norm.  Prints both figures."""
    elem_tol = tol if elem_tol is None else elem_tol
    rel, mx = rel_l2(got, want), max_abs_rel(got, want)
    print(f"{name} rel-L2 {rel:.2e}, max-abs / max {mx:.2e}")
    assert rel <= tol, f"{name} rel-L2 {rel:.3e} > {tol:g}"
    assert mx <= elem_tol, f"{name} max-abs error {mx:.3e} x max|want| > {elem_tol:g}"
    return rel, mx


def c1_case():
    cfg = synth.config(1)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(cfg, g, synth.phantom_seed(1))
    sino = synth.add_noise(synth.project(g, ell), cfg["noise_sigma"], synth.noise_seed(1))
    return cfg, g, sino.astype(np.float32)


def multipitch_case(endpoint_mode=0):
    """Config-1 scanner with a 150-slice volume: 2.6 pitches, so slices reuse
    the one-pitch tables with shifted views; ragged 61 x 45 xy grid."""
    cfg = dict(synth.config(1))
    cfg.update(nx=61, ny=45, nz=150, turns=5, endpoint_mode=endpoint_mode)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(dict(cfg, phantom="shepp_style"), g, 77)
    sino = synth.project(g, ell)
    return cfg, g, sino.astype(np.float32)


def fourpitch_case():
    """Config-1 scanner (58 slices per pitch) with a 194-slice volume on a ragged 61 x 45 grid:
    slices 0-19 lead four groups one pitch apart and slices 20-57 three, so the backprojection
    runs its four- and three-group forms with staged row bands, both with a partial last item."""
    cfg = dict(synth.config(1))
    cfg.update(nx=61, ny=45, nz=194, turns=6)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(dict(cfg, phantom="shepp_style"), g, 78)
    sino = synth.project(g, ell)
    return cfg, g, sino.astype(np.float32)


def finevoxel_case():
    """Config-1 scanner with 0.8 mm voxels on a 40 x 36 x 160 grid (60 slices per pitch, 2.7
    pitches): three- and two-group items whose row bands scale with the voxel size."""
    cfg = dict(synth.config(1))
    cfg.update(nx=40, ny=36, nz=160, turns=6, voxel=0.8)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(dict(cfg, phantom="shepp_style"), g, 79)
    sino = synth.project(g, ell)
    return cfg, g, sino.astype(np.float32)


def odd_case(tall=False):
    """Small geometry exercising every offset and parity: odd sizes, non-zero
    lambda0 / z0 / lambda_first / alpha and w offsets, odd n_psi, an axis voxel.  tall: a 69-column
    detector and 70 slices (22 per pitch), so that the slice-group backprojection takes four and
    three groups with row bands under all the offsets."""
    cfg = dict(R=300.0, D=620.0, views_per_turn=90, turns=4, n_rows=13, n_cols=53, n_cols_full=53, col_keep=1,
               det_half_width=21.0, nx=21, ny=17, nz=23, voxel=1.5, pitch_factor=1.0, n_psi=31)
    if tall:
        cfg.update(turns=8, n_cols=69, n_cols_full=69, det_half_width=27.0, nz=70)
    g = oracle.derive_geometry(cfg)
    g.update(lambda0=0.7, z0=-4.0, lambda_first=0.11, alpha_offset=0.25 * g["d_alpha"], w_offset=0.3 * g["d_w"])
    # re-centre the volume in the (shifted) scan, keep z_first on the slice grid
    dl = 2 * math.pi / g["views_per_turn"]
    h = g["P"] / (2 * math.pi)
    zc = g["z0"] + h * (g["lambda_first"] + 0.5 * g["n_views"] * dl)
    g["z_first"] = zc - 0.5 * (g["nz"] - 1) * g["dz"]
    rng = np.random.default_rng(15 if tall else 5)
    sino = rng.normal(size=(g["n_views"], g["n_rows"], g["n_cols"]))
    return cfg, g, sino.astype(np.float32)


def close_paths(a, b, name=""):
    """Two FP32 evaluations of the same operator whose slices were grouped differently (the
    multi-pitch kernel takes slices s, s + N, ... together where a launch holds them, so a slab
    launch and a whole-volume launch can group a slice differently): the geometry and end
    weights of a slice are then rounded relative to another reference view, and the results
    agree to FP32 rounding rather than bit for bit.  Bars: rel-L2 <= 2e-6 and every element
    within 1e-5 x max|b|; each path also meets the oracle bar in its own tests."""
    rel, mx = rel_l2(a, b), max_abs_rel(a, b)
    print(f"{name} paths: rel-L2 {rel:.2e}, max-abs / max {mx:.2e}")
    assert rel <= 2e-6 and mx <= 1e-5, (name, rel, mx)


def near_tie(frac, tol=1e-9):
    f = np.asarray(frac, dtype=np.float64)
    return (f < tol) | (f > 1 - tol)


def narrow_case():
    """Tiny scanner with a 9-column detector (narrower than any staged window)."""
    cfg = dict(R=100.0, D=200.0, views_per_turn=48, turns=3, n_rows=6, n_cols=9, n_cols_full=9, col_keep=1,
               det_half_width=4.0, nx=7, ny=5, nz=9, voxel=1.0, pitch_factor=1.0)
    g = oracle.derive_geometry(cfg)
    sino = np.random.default_rng(8).normal(size=(g["n_views"], g["n_rows"], g["n_cols"]))
    return cfg, g, sino.astype(np.float32)


def c3_small_case():
    """The differentiation scanner (config 3: every 2nd column of the clinical
    detector, 368 columns, 580 views/turn, 1.5 x max-fit pitch, rows truncated)
    with a 64 x 64 x 16 volume, so the oracle's transpose stays fast."""
    cfg = dict(synth.config(3))
    cfg.update(nx=64, ny=64, nz=16, turns=2)
    g = oracle.derive_geometry(cfg)
    return cfg, g


def rows80_case():
    """The config-1 scanner with 80 detector rows: a staged view window of 64 columns x 83 rows
    (21 KB) is too large for six ring slots at two CTAs per SM, so the backprojection runs with
    four slots (two slot pairs)."""
    cfg = dict(synth.config(1))
    cfg.update(n_rows=80)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(cfg, g, 81)
    sino = synth.project(g, ell)
    return cfg, g, sino.astype(np.float32)


def tall_case():
    """A detector of 264 rows and 33 columns: 528 kappa lines and 264 rows are more
    table entries than the rebinning kernels keep in shared memory, and more rows
    than the staged backprojection window holds, so the uncached table reads and
    the global-memory backprojection run."""
    cfg = dict(R=300.0, D=600.0, views_per_turn=64, turns=3, n_rows=264, n_cols=33, n_cols_full=33, col_keep=1,
               det_half_width=8.0, nx=12, ny=12, nz=10, voxel=1.0, pitch_factor=1.0)
    g = oracle.derive_geometry(cfg)
    sino = np.random.default_rng(9).normal(size=(g["n_views"], g["n_rows"], g["n_cols"]))
    return cfg, g, sino.astype(np.float32)
