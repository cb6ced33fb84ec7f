"""Pins of the oracle's PI-window discretisation and of its extents (Eq. (maxvalue)).

Each check compares the oracle with something it does not compute itself: the
closed-form PI line of a point on the axis (a diameter, so lam_i, lam_o = zeta -+ pi/2),
the identity that the end weights of the midpoint rule integrate the PI interval
exactly, the hard indicator's definition, and the Tam-Danielsson window that bounds
every projection a voxel backprojects.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from cases import odd_case


def axis_geometry(nz=9, vpt=128, endpoint_mode=0):
    """Config-1 scanner with a one-voxel-wide column on the axis (x = y = 0)."""
    cfg = dict(synth.config(1))
    cfg.update(nx=1, ny=1, nz=nz, views_per_turn=vpt, endpoint_mode=endpoint_mode)
    g = oracle.derive_geometry(cfg)
    assert g["x0"] == 0.0 and g["y0"] == 0.0
    return g


def axis_windows(g):
    """Closed-form PI interval and midpoint-rule view window of the axis voxel of each
    table slice: lam_i, lam_o = zeta -+ pi/2 with zeta = (z - z0) / h."""
    N = oracle.pitch_slices(g)
    h = g["P"] / (2 * math.pi)
    dl = 2 * math.pi / g["views_per_turn"]
    z = g["z_first"] + np.arange(N) * g["dz"]
    zeta = (z - g["z0"]) / h
    li, lo = zeta - math.pi / 2, zeta + math.pi / 2
    ui, uo = (li - g["lambda_first"]) / dl, (lo - g["lambda_first"]) / dl
    k0 = np.floor(ui).astype(np.int64)
    k1 = (np.ceil(uo) - 1).astype(np.int64)
    return zeta, li, lo, k0, k1, h, dl


@pytest.mark.parametrize("which", ["c1", "odd"])
def test_end_weights_integrate_the_pi_interval(which):
    # Midpoint rule over [lam_i, lam_o] (reading of the PI-window discretisation): the weights
    # of the views that touch the interval sum to its length, sum_k omega_k dl = lam_o - lam_i.
    # A complemented end weight (u - floor u for its complement) breaks this by up to 2 dl.
    g = oracle.derive_geometry(synth.config(1)) if which == "c1" else odd_case()[1]
    t = oracle.pi_table(g)
    dl = 2 * math.pi / g["views_per_turn"]
    assert (t["k1"] > t["k0"]).all()
    total = (t["w0"] + t["w1"] + (t["k1"] - t["k0"] - 1)) * dl
    assert np.abs(total - (t["lam_o"] - t["lam_i"])).max() < 1e-12
    assert (t["w0"] > 0).all() and (t["w0"] <= 1).all() and (t["w1"] > 0).all() and (t["w1"] <= 1).all()
    # the first and last views are the ones whose arcs [l_k, l_k+1] contain the endpoints
    lam = lambda k: g["lambda_first"] + k * dl  # noqa: E731
    assert (lam(t["k0"]) <= t["lam_i"]).all() and (t["lam_i"] < lam(t["k0"] + 1)).all()
    assert (lam(t["k1"]) < t["lam_o"]).all() and (t["lam_o"] <= lam(t["k1"] + 1)).all()


def test_hard_endpoints_take_the_views_whose_centre_is_inside():
    # endpoint_mode 1: the hard indicator of the paper's integral, views with l_{k+1/2} in
    # [lam_i, lam_o], weight 1
    cfg = dict(synth.config(1))
    cfg.update(endpoint_mode=1, nx=24, ny=20, nz=8)
    g = oracle.derive_geometry(cfg)
    t = oracle.pi_table(g)
    dl = 2 * math.pi / g["views_per_turn"]
    mid = lambda k: g["lambda_first"] + (k + 0.5) * dl  # noqa: E731
    assert (mid(t["k0"]) >= t["lam_i"]).all() and (mid(t["k0"] - 1) < t["lam_i"]).all()
    assert (mid(t["k1"]) <= t["lam_o"]).all() and (mid(t["k1"] + 1) > t["lam_o"]).all()
    assert (t["w0"] == 1).all() and (t["w1"] == 1).all()


@pytest.mark.parametrize("vpt", [128, 97])
def test_extents_and_update_count_on_axis_closed_form(vpt):
    # A column on the axis: alpha* = 0 in every view, v* = R, and w* = (D h / R)(zeta - lam), so
    # Eq. (maxvalue)'s extents over the voxels' own views (at the half-view angles l_{k+1/2}) are
    # closed forms of the axis PI intervals.  Taking the views at l_k instead, or over the
    # union window of the slices, moves w_min / w_max by at least (D h / R) dl / 2.
    g = axis_geometry(vpt=vpt)
    zeta, li, lo, k0, k1, h, dl = axis_windows(g)
    pl = oracle.Plan(g)
    assert np.array_equal(pl.pi["k0"][:, 0, 0], k0) and np.array_equal(pl.pi["k1"][:, 0, 0], k1)
    ext = pl.extents()
    s = g["D"] * h / g["R"]
    w_first = s * (zeta - (g["lambda_first"] + (k0 + 0.5) * dl))  # w* of each slice's first view
    w_last = s * (zeta - (g["lambda_first"] + (k1 + 0.5) * dl))
    assert abs(ext[0] - li.min()) < 1e-12 and abs(ext[1] - lo.max()) < 1e-12
    assert ext[2] == 0.0 and ext[3] == 0.0
    assert abs(ext[5] - w_first.max()) < 1e-9 and abs(ext[4] - w_last.min()) < 1e-9
    # the window is exactly pi wide: vpt / 2 views cover it, one more unless an endpoint
    # falls on a view boundary; every slice of the column counts once per pitch it repeats in
    N = oracle.pitch_slices(g)
    per_slice = k1 - k0 + 1
    assert set(per_slice.tolist()) <= {math.ceil(vpt / 2), math.ceil(vpt / 2) + 1}
    reps = np.array([(g["nz"] - 1 - j) // N + 1 if j < g["nz"] else 0 for j in range(N)])
    assert pl.update_count() == int((reps * per_slice).sum())


def test_extents_lambda_are_the_pointwise_pi_endpoints():
    # lam_min / lam_max of Eq. (maxvalue) over one pitch are the extremes of the PI endpoints
    # of its voxels, each solved on its own (the solver is pinned by the axis closed form,
    # collinearity and the TD identities)
    _, g, _ = odd_case()
    pl = oracle.Plan(g)
    ext = pl.extents()
    N = oracle.pitch_slices(g)
    li, lo = [], []
    for j in range(N):
        z = g["z_first"] + j * g["dz"]
        for iy in range(g["ny"]):
            for ix in range(g["nx"]):
                a, b = oracle.pi_endpoints(g, g["x0"] + ix * g["dx"], g["y0"] + iy * g["dy"], z)
                li.append(a)
                lo.append(b)
    assert ext[0] == min(li) and ext[1] == max(lo)


def small_c1():
    cfg = dict(synth.config(1))
    cfg.update(nx=8, ny=6, nz=4)
    return oracle.derive_geometry(cfg)


@pytest.mark.parametrize("which", ["c1", "odd"])
def test_extents_are_over_each_voxels_own_views_inside_the_td_window(which):
    # Eq. (maxvalue) read as the extremes of (alpha*, w*) over the views each voxel of one pitch
    # backprojects, at the half-view angles l_{k+1/2}.  Brute force over every voxel and view of
    # a small volume: each projection lies inside the Tam-Danielsson window w_bot(alpha*) <= w*
    # <= w_top(alpha*) up to the half view by which the end views reach past lam_i / lam_o
    # (bounded per voxel by how far w* leaves the boundary within half a view of it), and the extents are exactly
    # the extremes of these projections.  Extents over the union window of a slice, or at l_k,
    # fail one of the two.
    g = small_c1() if which == "c1" else odd_case()[1]
    pl = oracle.Plan(g)
    ext = pl.extents()
    t = pl.pi
    N = oracle.pitch_slices(g)
    dl = 2 * math.pi / g["views_per_turn"]
    lam = lambda k: g["lambda_first"] + (k + 0.5) * dl  # noqa: E731
    amin = wmin = math.inf
    amax = wmax = -math.inf
    for j in range(N):
        z = g["z_first"] + j * g["dz"]
        for iy in range(g["ny"]):
            for ix in range(g["nx"]):
                x, y = g["x0"] + ix * g["dx"], g["y0"] + iy * g["dy"]
                li, lo = t["lam_i"][j, iy, ix], t["lam_o"][j, iy, ix]
                # slack: how far w* leaves its TD boundary within half a view of each endpoint
                slack = 0.0
                for le, bound in ((li, oracle.w_td_top), (lo, oracle.w_td_bottom)):
                    for d in (-0.5 * dl, 0.5 * dl):
                        a, w, _ = oracle.project_point(g, le + d, x, y, z)
                        slack = max(slack, abs(w - bound(g, a)))
                for k in range(t["k0"][j, iy, ix], t["k1"][j, iy, ix] + 1):
                    a, w, _ = oracle.project_point(g, lam(k), x, y, z)
                    assert oracle.w_td_bottom(g, a) - slack - 1e-9 <= w <= oracle.w_td_top(g, a) + slack + 1e-9
                    amin, amax, wmin, wmax = min(amin, a), max(amax, a), min(wmin, w), max(wmax, w)
    assert np.allclose(ext[2:], [amin, amax, wmin, wmax], rtol=0, atol=1e-12)
