"""Pins of the oracle's filter steps (Sec. II steps 1-6) against closed forms."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def g1():
    return oracle.derive_geometry(synth.config(1))


def grids(g):
    lam = g["lambda_first"] + np.arange(g["n_views"]) * 2 * math.pi / g["views_per_turn"]
    alpha = (np.arange(g["n_cols"]) - 0.5 * (g["n_cols"] - 1)) * g["d_alpha"] + g["alpha_offset"]
    w = (np.arange(g["n_rows"]) - 0.5 * (g["n_rows"] - 1)) * g["d_w"] + g["w_offset"]
    return lam, alpha, w


def test_derivative_exact_on_quadratics(g1):
    # d/dq + d/dalpha at fixed w (Eq. (Deriv)); the 2x2 centred stencil is exact
    # for every polynomial of degree 2 in (lambda, alpha) at the cell centre.
    g = dict(g1)
    g["n_views"] = 6
    lam, alpha, w = grids(g)
    L, W, A = np.meshgrid(lam, w, alpha, indexing="ij")
    c = np.random.default_rng(1).normal(size=7)
    f = c[0] * L * L + c[1] * A * A + c[2] * L * A + c[3] * L + c[4] * A + c[5] * W * L + c[6] * W * A
    g1v = oracle.derivative(g, f)
    Lh = 0.5 * (L[1:, :, 1:] + L[:-1, :, :-1])
    Ah = 0.5 * (A[1:, :, 1:] + A[:-1, :, :-1])
    Wh = W[1:, :, 1:]
    want = (2 * c[0] * Lh + c[2] * Ah + c[3] + c[5] * Wh) + (2 * c[1] * Ah + c[2] * Lh + c[4] + c[6] * Wh)
    assert np.max(np.abs(g1v - want)) < 1e-7 * np.max(np.abs(want))


def test_length_weight(g1):
    g = dict(g1)
    x = np.ones((2, g["n_rows"], g["n_cols"] - 1))
    y = oracle.length_weight(g, x)
    _, _, w = grids(g)
    # D / |ray to (0, w)| = cos of the cone angle of row w
    assert np.allclose(y[1, :, 5], np.cos(np.arctan(w / g["D"])), rtol=1e-14)


def _half_period_geometry(nc):
    g = oracle.derive_geometry(synth.config(1))
    g = dict(g)
    g["n_cols"] = nc
    g["d_alpha"] = math.pi / (nc - 1)  # columns span [-pi/2, pi/2]
    return g


@pytest.mark.parametrize("nc", [513, 1025])
def test_hilbert_closed_form_pairs(nc):
    # With h_H(s) = 1/(pi s), the transform over (-pi/2, pi/2) at constant psi
    # (Eq. (HF)) maps cos -> sin and sin -> -cos (t = tan(alpha) turns it into
    # the line Hilbert transform of 1/(1+t^2) and t/(1+t^2)).
    g = _half_period_geometry(nc)
    half = (np.arange(nc - 1) + 0.5 - 0.5 * (nc - 1)) * g["d_alpha"]
    full = (np.arange(nc) - 0.5 * (nc - 1)) * g["d_alpha"]
    g3 = np.stack([np.cos(half), np.sin(half)])[None]
    g4 = oracle.hilbert(g, g3)[0]
    inner = np.abs(full) < 1.3
    err_cos = np.max(np.abs(g4[0] - np.sin(full))[inner])
    err_sin = np.max(np.abs(g4[1] + np.cos(full))[inner])
    tol = 2.0 * g["d_alpha"] ** 2 + 1e-3 * (g["d_alpha"] / (math.pi / 512)) ** 2
    assert err_cos < tol and err_sin < tol
    # a half-sample shift of the kernel would leave an O(d_alpha) error
    assert err_cos < 0.05 * g["d_alpha"]


def test_forward_rebin_linear_in_w(g1):
    # Linear interpolation in w is exact for data linear in w (Eq. (FR)).
    kap = oracle.kappa_table(g1)
    _, alpha, w = grids(g1)
    g2 = np.broadcast_to((0.7 + 0.03 * w)[None, :, None], (2, g1["n_rows"], g1["n_cols"] - 1))
    g3 = oracle.forward_rebin(g1, kap, g2)
    am = oracle.alpha_m(g1)
    npsi = oracle.n_psi(g1)
    psi = -(math.pi / 2 + am) + np.arange(npsi) * 2 * (math.pi / 2 + am) / (npsi - 1)
    ah = 0.5 * (alpha[1:] + alpha[:-1])
    for l in range(0, npsi, 7):
        for c in range(0, g1["n_cols"] - 1, 9):
            wk = oracle.w_kappa(g1, ah[c], psi[l])
            if w[0] <= wk <= w[-1]:
                assert g3[1, l, c] == pytest.approx(0.7 + 0.03 * wk, rel=1e-12)


def test_backward_rebin_linear_in_psi(g1):
    psit = oracle.psi_table(g1)
    npsi = oracle.n_psi(g1)
    am = oracle.alpha_m(g1)
    psi = -(math.pi / 2 + am) + np.arange(npsi) * 2 * (math.pi / 2 + am) / (npsi - 1)
    g4 = np.broadcast_to((1.0 - 0.2 * psi)[None, :, None], (1, npsi, g1["n_cols"]))
    g5 = oracle.backward_rebin(g1, psit, g4)
    _, alpha, w = grids(g1)
    for r in range(0, g1["n_rows"], 3):
        for c in range(0, g1["n_cols"], 11):
            p = oracle.psi_hat(g1, alpha[c], w[r])
            if p is None:
                # no kappa-line reaches this sample: it lies outside every line's span
                pm = math.pi / 2 + am
                span = [oracle.w_kappa(g1, alpha[c], q) for q in np.linspace(-pm, pm, 2001)]
                assert not (min(span) <= w[r] <= max(span)) and g5[0, r, c] == 0.0
                continue
            assert g5[0, r, c] == pytest.approx(1.0 - 0.2 * p, rel=1e-12)


def test_post_cosine(g1):
    _, alpha, _ = grids(g1)
    y = oracle.post_cosine(g1, np.ones((1, g1["n_rows"], g1["n_cols"])))
    assert np.allclose(y[0, 3], np.cos(alpha), rtol=1e-15)


def test_filter_is_composition(g1):
    rng = np.random.default_rng(2)
    sino = rng.normal(size=(5, g1["n_rows"], g1["n_cols"]))
    pl = oracle.Plan(g1, with_pi=False)
    gF = pl.filter(sino)
    steps = oracle.post_cosine(g1, oracle.backward_rebin(g1, pl.psi, oracle.hilbert(
        g1, oracle.forward_rebin(g1, pl.kap, oracle.length_weight(g1, oracle.derivative(g1, sino))))))
    assert np.allclose(gF, steps, rtol=1e-13, atol=1e-13)
