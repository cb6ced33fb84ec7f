"""Pins of the oracle's geometry (PI-lines, kappa-lines, TD window) against
facts the paper and the geometry fix independently of the oracle's formulas."""
import math

import numpy as np
import pytest

import oracle
import synth


def helix(g, lam):
    ph = lam + g["lambda0"]
    return np.array([g["R"] * math.cos(ph), g["R"] * math.sin(ph), g["z0"] + g["P"] * lam / (2 * math.pi)])


@pytest.fixture(scope="module")
def g1():
    g = oracle.derive_geometry(synth.config(1))
    g["lambda0"] = 0.37  # non-zero start angle exercises every l0 term
    g["z0"] = -3.0
    return g


@pytest.fixture(scope="module")
def g2():
    return oracle.derive_geometry(synth.config(2))


def random_points(g, n, seed, rmax_frac=0.95):
    rng = np.random.default_rng(seed)
    r = rmax_frac * g["R"] * np.sqrt(rng.uniform(size=n))
    th = rng.uniform(0, 2 * math.pi, size=n)
    z = rng.uniform(-200, 200, size=n)
    return np.stack([r * np.cos(th), r * np.sin(th), z], 1)


def test_pi_on_axis_closed_form(g1):
    # On the axis every chord through x is a diameter: d = pi/2, b = (z - z0)/h.
    h = g1["P"] / (2 * math.pi)
    for z in (-50.0, 0.0, 13.3, 400.0):
        li, lo = oracle.pi_endpoints(g1, 0.0, 0.0, z)
        zeta = (z - g1["z0"]) / h
        assert abs(li - (zeta - math.pi / 2)) < 1e-12
        assert abs(lo - (zeta + math.pi / 2)) < 1e-12


@pytest.mark.parametrize("which", ["g1", "g2"])
def test_pi_line_collinear(which, request):
    # The PI-line is the chord a(l_i) -- a(l_o) through x with l_o - l_i < 2 pi.
    g = request.getfixturevalue(which)
    for x in random_points(g, 60, seed=5):
        li, lo = oracle.pi_endpoints(g, *x)
        assert 0.0 < lo - li < 2 * math.pi
        ai, ao = helix(g, li), helix(g, lo)
        seg = ao - ai
        t = np.dot(x - ai, seg) / np.dot(seg, seg)
        assert 0.0 < t < 1.0
        dist = np.linalg.norm(x - (ai + t * seg))
        assert dist < 1e-9 * g["R"]


def test_pi_endpoints_on_td_boundaries(g1, g2):
    # Seen from a(l_i) (resp. a(l_o)) the point x lies on the upper (lower)
    # Tam-Danielsson boundary, the projection of the next (previous) helix turn.
    for g in (g1, g2):
        for x in random_points(g, 40, seed=7, rmax_frac=0.9):
            li, lo = oracle.pi_endpoints(g, *x)
            a, w, _ = oracle.project_point(g, li, *x)
            assert abs(w - oracle.w_td_top(g, a)) < 1e-9 * max(1.0, abs(w))
            a, w, _ = oracle.project_point(g, lo, *x)
            assert abs(w - oracle.w_td_bottom(g, a)) < 1e-9 * max(1.0, abs(w))


def test_periodicity(g1):
    # Sec. II periodic properties: l_{i,o}(x + kP e_z) = l_{i,o}(x) + 2 pi k;
    # v*, alpha*, w* invariant under (l + 2 pi k, x + kP e_z).
    for x in random_points(g1, 20, seed=9):
        li, lo = oracle.pi_endpoints(g1, *x)
        for k in (-2, 1, 3):
            xk = x + np.array([0, 0, k * g1["P"]])
            lik, lok = oracle.pi_endpoints(g1, *xk)
            assert abs(lik - (li + 2 * math.pi * k)) < 1e-11
            assert abs(lok - (lo + 2 * math.pi * k)) < 1e-11
            lam = 0.5 * (li + lo)
            p0 = np.array(oracle.project_point(g1, lam, *x))
            pk = np.array(oracle.project_point(g1, lam + 2 * math.pi * k, *xk))
            assert np.allclose(p0, pk, rtol=1e-11, atol=1e-11)


def test_pi_endpoints_increase_with_z(g1):
    # Along a line parallel to the axis the PI-line's endpoints move up the helix with
    # the point: l_i(z) and l_o(z) are strictly increasing (the PI window shifts
    # monotonically, the property the backprojection's window ramps use).  The sweep
    # spans more than a pitch, so the one-turn jump of the periodic property is crossed.
    for x in random_points(g1, 12, seed=21):
        zs = x[2] + np.linspace(-0.7, 0.7, 57) * g1["P"]
        ends = np.array([oracle.pi_endpoints(g1, x[0], x[1], z) for z in zs])
        assert np.all(np.diff(ends[:, 0]) > 0) and np.all(np.diff(ends[:, 1]) > 0)


def test_pi_table_windows_monotone_in_slice(g1):
    # the same property on the table: window start k0 - w0 and end k1 + w1 (view
    # units) never decrease from slice to slice, including slice N-1 -> slice 0 of
    # the next pitch one turn later
    t = oracle.pi_table(g1)
    vpt = g1["views_per_turn"]
    s = t["k0"] - t["w0"]
    e = t["k1"] + t["w1"]
    s = np.concatenate([s, s[:1] + vpt], 0)
    e = np.concatenate([e, e[:1] + vpt], 0)
    assert np.all(np.diff(s, axis=0) >= 0) and np.all(np.diff(e, axis=0) >= 0)


def test_project_point_matches_acquisition_rays(g1):
    # The ray the acquisition model fires at detector (alpha*, w*) passes through x.
    for x in random_points(g1, 30, seed=11, rmax_frac=0.8):
        for lam in (0.3, 2.0, 5.5):
            a, w, v = oracle.project_point(g1, lam, *x)
            s, d = synth.ray(g1, lam, a, w)
            t = np.dot(x - s, d)
            assert np.linalg.norm(x - (s + t * d)) < 1e-9 * g1["R"]
            # v* is the distance along the central ray direction e_v
            ph = lam + g1["lambda0"]
            ev = np.array([-math.cos(ph), -math.sin(ph), 0.0])
            assert abs(np.dot(x - s, ev) - v) < 1e-9 * g1["R"]


def test_kappa_line_lies_in_kappa_plane(g2):
    # A kappa-plane contains a(l), a(l + psi), a(l + 2 psi); its intersection with
    # the detector is w = w_kappa(alpha, psi).  Every such ray lies in the plane.
    rng = np.random.default_rng(3)
    am = oracle.alpha_m(g2)
    for _ in range(60):
        lam = rng.uniform(0, 20)
        psi = rng.uniform(-math.pi / 2 - am, math.pi / 2 + am)
        if abs(psi) < 1e-3:
            continue
        alpha = rng.uniform(-am, am)
        w = oracle.w_kappa(g2, alpha, psi)
        s, d = synth.ray(g2, lam, alpha, w)
        a0, a1, a2 = helix(g2, lam), helix(g2, lam + psi), helix(g2, lam + 2 * psi)
        n = np.cross(a1 - a0, a2 - a0)
        n /= np.linalg.norm(n)
        assert abs(np.dot(n, d)) < 1e-10
        assert np.linalg.norm(s - a0) < 1e-9


def test_td_boundaries_are_extreme_kappa_lines(g1, g2):
    for g in (g1, g2):
        for a in np.linspace(-oracle.alpha_m(g), oracle.alpha_m(g), 9):
            assert oracle.w_kappa(g, a, math.pi / 2 - a) == pytest.approx(oracle.w_td_top(g, a), rel=1e-12)
            assert oracle.w_kappa(g, a, -math.pi / 2 - a) == pytest.approx(oracle.w_td_bottom(g, a), rel=1e-12)


def test_fit_pitch_fills_detector_and_envelope(g1, g2):
    # At the unrounded max-fit pitch the widest TD extent (and every kappa-line
    # of the rebinning range) reaches exactly the outermost row centre.
    for g in (g1, g2):
        am = oracle.alpha_m(g)
        gg = dict(g)
        gg["P"] = oracle.fit_pitch(g["R"], g["D"], g["n_rows"], g["d_w"], am)
        top = 0.5 * (g["n_rows"] - 1) * g["d_w"]
        alphas = np.linspace(-am, am, 401)
        td = max(max(oracle.w_td_top(gg, a), -oracle.w_td_bottom(gg, a)) for a in alphas)
        assert td == pytest.approx(top, rel=1e-12)
        pm = math.pi / 2 + am
        env = max(abs(oracle.w_kappa(gg, a, p)) for a in alphas[::20] for p in np.linspace(-pm, pm, 1501))
        assert env <= top * (1 + 1e-12)
        assert env >= top * (1 - 1e-6)


def test_derived_geometry_values():
    # The workloads' derived values: alpha_m, pitch, slices per pitch.
    g = oracle.derive_geometry(synth.config(1))
    assert oracle.alpha_m(g) == pytest.approx(math.asin(32 * math.sqrt(2) / 500), rel=1e-15)
    assert g["P"] == 58.0 and oracle.pitch_slices(g) == 58 and g["d_w"] == 2.0
    g = oracle.derive_geometry(synth.config(2))
    assert g["P"] == 70.0 and oracle.pitch_slices(g) == 70
    g = oracle.derive_geometry(synth.config(3))
    assert g["P"] == 150.0


def _brute_psi_hat(g, alpha, w, n=4000):
    pm = math.pi / 2 + oracle.alpha_m(g)
    best = None
    for side in (1.0, -1.0):
        ps = side * np.linspace(0.0, pm, n + 1)
        f = np.array([oracle.w_kappa(g, alpha, p) - w for p in ps])
        sgn = np.sign(f)
        ch = np.nonzero(sgn[1:] * sgn[:-1] <= 0)[0]
        if ch.size:
            p = 0.5 * (ps[ch[0]] + ps[ch[0] + 1])
            if best is None or abs(p) < abs(best):
                best = p
    return best, pm / n


def test_psi_hat_smallest_root_matches_dense_scan(g2):
    # Config-2 fan (alpha_m = 0.654) has a non-monotone branch; the rule is the
    # root of smallest |psi| (Sec. II, backward height rebinning).
    rng = np.random.default_rng(21)
    am = oracle.alpha_m(g2)
    top = 0.5 * (g2["n_rows"] - 1) * g2["d_w"]
    cases = [(am * 0.999, 0.99 * oracle.w_kappa(g2, am * 0.999, 1.42)),
             (-am * 0.999, -0.99 * oracle.w_kappa(g2, am * 0.999, 1.42))]
    cases += [(rng.uniform(-am, am), rng.uniform(-1.1 * top, 1.1 * top)) for _ in range(40)]
    for alpha, w in cases:
        ref, step = _brute_psi_hat(g2, alpha, w)
        got = oracle.psi_hat(g2, alpha, w)
        if ref is None:
            assert got is None
        else:
            assert got is not None and abs(got - ref) <= step
            assert oracle.w_kappa(g2, alpha, got) == pytest.approx(w, abs=1e-9)


def test_psi_hat_round_trip(g1):
    am = oracle.alpha_m(g1)
    for a in np.linspace(-am, am, 7):
        for p in np.linspace(-1.4, 1.4, 15):
            assert oracle.psi_hat(g1, a, oracle.w_kappa(g1, a, p)) == pytest.approx(p, abs=1e-12)
