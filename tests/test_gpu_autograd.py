"""Differentiation: the autograd layer's backward is the hand-written adjoint.

Checked against (1) the FP64 oracle's transpose on the config-3 scanner
(sparse 368-column detector, 1.5 x max-fit pitch), (2) central finite
differences along random directions supported on 16 x 16 x 8 sub-volumes of
the cotangent (exact for a linear map up to FP32 rounding), (3) the dot-product
identity on batch 4.
"""
import numpy as np
import pytest

import oracle
from cases import c3_small_case, check32, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as kats
    from paper_2201_02309_b300.autograd import KatsevichFunction, KatsevichLayer
    return torch, kats, KatsevichFunction, KatsevichLayer


def test_backward_matches_oracle_transpose(env):
    torch, kats, Fn, Layer = env
    _, g = c3_small_case()
    layer = Layer(g)
    rng = np.random.default_rng(0)
    sino = torch.from_numpy(rng.normal(size=layer.plan.sino_shape).astype(np.float32)).cuda().requires_grad_(True)
    cot = np.zeros(layer.plan.vol_shape, np.float32)
    cot[4:12, 20:36, 24:40] = rng.normal(size=(8, 16, 16))
    vol = layer(sino)
    vol.backward(torch.from_numpy(cot).cuda())
    op = oracle.Plan(g)
    want = op.adjoint(cot.astype(np.float64))
    check32(sino.grad.cpu().numpy(), want)
    check32(vol.detach().cpu().numpy(), op.recon(sino.detach().cpu().numpy().astype(np.float64)))


def test_adjoint_halves_match_oracle(env):
    # localises the transpose's error: step 7^T and steps 1-6^T separately
    torch, kats, Fn, Layer = env
    _, g = c3_small_case()
    plan = kats.Plan(g)
    op = oracle.Plan(g)
    rng = np.random.default_rng(3)
    cot = np.zeros(plan.vol_shape, np.float32)
    cot[4:12, 20:36, 24:40] = rng.normal(size=(8, 16, 16))
    v0, nv = plan.info["first_view"], plan.info["n_filtered_views"]
    gfa = plan.backproject_adjoint(torch.from_numpy(cot).cuda()).cpu().numpy()
    want = op.backproject_adjoint(cot.astype(np.float64), v0, nv)
    err_bp = rel_l2(gfa[..., :g["n_cols"]], want)
    sa = plan.filter_adjoint(torch.from_numpy(np.ascontiguousarray(gfa)).cuda()).cpu().numpy()
    gf64 = gfa[..., :g["n_cols"]].astype(np.float64)
    full = np.zeros((g["n_views"] - 1,) + gf64.shape[1:])
    full[v0:v0 + nv] = gf64
    want_f = op.filter_adjoint(full)
    err_f = rel_l2(sa, want_f)
    print(f"step 7^T rel-L2 {err_bp:.2e}, steps 1-6^T rel-L2 {err_f:.2e}")
    assert err_bp < 1e-5
    assert err_f < 1e-5


def test_finite_differences_on_subvolumes(env):
    torch, kats, Fn, Layer = env
    _, g = c3_small_case()
    plan = kats.Plan(g)
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.normal(size=plan.sino_shape).astype(np.float32)).cuda().requires_grad_(True)
    for trial in range(3):
        u = np.zeros(plan.vol_shape, np.float32)
        z0, y0, x0 = rng.integers(0, 8), rng.integers(0, 48), rng.integers(0, 48)
        u[z0:z0 + 8, y0:y0 + 16, x0:x0 + 16] = rng.normal(size=(8, 16, 16))
        ut = torch.from_numpy(u).cuda()
        x.grad = None
        (Fn.apply(x, plan) * ut).sum().backward()
        v = torch.from_numpy(rng.normal(size=plan.sino_shape).astype(np.float32)).cuda()
        eps = 1e-2 * float(x.detach().abs().max())
        with torch.no_grad():
            fp = (Fn.apply(x + eps * v, plan).double() * ut.double()).sum()
            fm = (Fn.apply(x - eps * v, plan).double() * ut.double()).sum()
        fd = float((fp - fm) / (2 * eps))
        an = float((x.grad.double() * v.double()).sum())
        assert abs(fd - an) <= 2e-3 * max(abs(an), 1e-6), (trial, fd, an)


def test_dot_product_batch4(env):
    torch, kats, Fn, Layer = env
    _, g = c3_small_case()
    plan = kats.Plan(g)
    rng = np.random.default_rng(2)
    xb = torch.from_numpy(rng.normal(size=(4,) + plan.sino_shape).astype(np.float32)).cuda()
    yb = torch.from_numpy(rng.normal(size=(4,) + plan.vol_shape).astype(np.float32)).cuda()
    ax = plan.recon(xb)
    aty = plan.adjoint(yb)
    for b in range(4):
        lhs = float((ax[b].double() * yb[b].double()).sum())
        rhs = float((xb[b].double() * aty[b].double()).sum())
        assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


def test_reduced_precision_forward_fp32_backward(env):
    """A BF16 / FP16 forward differentiates through the FP32 transpose."""
    torch, kats, Fn, Layer = env
    _, g = c3_small_case()
    rng = np.random.default_rng(3)
    cot = np.zeros(kats.Plan(g).vol_shape, np.float32)
    cot[4:12, 20:36, 24:40] = rng.normal(size=(8, 16, 16))
    op = oracle.Plan(g)
    want = op.adjoint(cot.astype(np.float64))
    for prec in (kats.KATS_PREC_BF16, kats.KATS_PREC_FP16):
        layer = Layer(g, precision=prec)
        sino = torch.from_numpy(rng.normal(size=layer.plan.sino_shape).astype(np.float32)).cuda().requires_grad_(True)
        vol = layer(sino)
        # the forward is the reduced form itself (its accuracy is gated on phantoms elsewhere)
        assert torch.equal(vol.detach(), layer.plan.recon(sino.detach(), precision=prec))
        vol.backward(torch.from_numpy(cot).cuda())
        check32(sino.grad.cpu().numpy(), want)
