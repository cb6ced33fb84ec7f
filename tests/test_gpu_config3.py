"""The differentiation workload at its stated size: the clinical scanner's detector with every
2nd column (368) or every 4th (184), 580 views/turn, 4 turns, 1.5 x max-fit pitch (rows
truncated), a 256 x 256 x 64 volume, batch 4 (the paper's sparse-detector data, Sec. III-C).

* kappa / psi_hat integer tables bit for bit against the oracle (alpha_m = 0.31);
* the forward operator on sampled voxels of each batch item against the oracle's chain;
* the transpose on cotangents supported on 16 x 16 x 8 sub-volumes against the oracle's
  transpose: step 7's transpose over the sub-volume's own voxels (the oracle builds the
  PI windows of exactly those voxels) followed by the transpose of steps 1-6 on the
  scanner's full tables; every sinogram entry compared;
* the dot-product identity <A x, y> = <x, A^T y> on batch 4.
"""
import numpy as np
import pytest

import oracle
import synth
from cases import check32, near_tie

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as kats
    return torch, kats


def geometry(keep):
    cfg = dict(synth.config(3))
    cfg.update(n_cols=736 // keep, col_keep=keep)
    return oracle.derive_geometry(cfg)


@pytest.fixture(scope="module", params=[2, 4], ids=["cols368", "cols184"])
def c3(env, request):
    torch, kats = env
    g = geometry(request.param)
    assert (g["nx"], g["ny"], g["nz"], g["views_per_turn"], g["P"]) == (256, 256, 64, 580, 150.0)
    return g, kats.Plan(g), oracle.Plan(g, with_pi=False)


def test_c3_kappa_psi_tables(c3):
    g, kp, op = c3
    for name, (idx, frac) in (("kappa", op.kap), ("psi", op.psi)):
        got = kp.table(f"{name}_idx")
        bad = got != idx
        assert not (bad & ~near_tie(frac)).any(), f"{name}: {int((bad & ~near_tie(frac)).sum())} mismatches"
        print(f"{name}_idx {got.shape}: {int(bad.sum())} mismatches, {int(near_tie(frac).sum())} near-ties")
        same = ~bad
        assert np.abs(kp.table(f"{name}_frac") - frac)[same].max() < 2e-7


def test_c3_forward_batch4_sampled(env, c3):
    torch, kats = env
    g, kp, op = c3
    rng = np.random.default_rng(31)
    x = rng.normal(size=(4,) + kp.sino_shape).astype(np.float32)
    vol = kp.recon(torch.from_numpy(x).cuda()).cpu().numpy()
    n = 120
    ijk = np.stack([rng.integers(0, 256, n), rng.integers(0, 256, n), rng.integers(0, 64, n)], 1)
    ijk[:4] = [(0, 0, 0), (255, 0, 63), (0, 255, 31), (255, 255, 32)]
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    v0, v1 = int(ka.min()), int(kb.max())
    for b in range(4):
        gF = op.filter(x[b].astype(np.float64), v0, v1 - v0 + 1)
        want = oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb))
        check32(vol[b][ijk[:, 2], ijk[:, 1], ijk[:, 0]], want, name=f"item {b}")


def sub_geometry(g, ox, oy, oz, size=(16, 16, 8)):
    """The same scan with only the voxels [oz:oz+8, oy:oy+16, ox:ox+16] of the volume."""
    s = dict(g)
    s.update(nx=size[0], ny=size[1], nz=size[2], x0=g["x0"] + ox * g["dx"], y0=g["y0"] + oy * g["dy"],
             z_first=g["z_first"] + oz * g["dz"])
    return s


def oracle_adjoint_subvolume(g, op, y_sub, ox, oy, oz):
    """A^T y for a cotangent y supported on one sub-volume: step 7^T over that sub-volume's
    voxels (their own PI windows), then steps 1-6^T with the scanner's tables."""
    gs = sub_geometry(g, ox, oy, oz)
    ps = oracle.Plan(gs)
    nv = g["n_views"] - 1
    gF_adj = ps.backproject_adjoint(y_sub.astype(np.float64), 0, nv)
    # steps 1-6^T of the views the sub-volume reached (filtered view k feeds sinogram views k, k+1)
    hit = np.flatnonzero(np.abs(gF_adj).reshape(nv, -1).max(1) > 0)
    a, b = int(hit[0]), int(hit[-1])
    out = np.zeros((g["n_views"],) + gF_adj.shape[1:])
    out[a:b + 2] = op.filter_adjoint(gF_adj[a:b + 1])
    return out


def test_c3_adjoint_subvolume_cotangents_batch4(env, c3):
    torch, kats = env
    g, kp, op = c3
    rng = np.random.default_rng(32)
    y = np.zeros((4,) + kp.vol_shape, np.float32)
    corners = [(0, 0, 0), (240, 240, 56), (120, 7, 30), (37, 200, 13)]
    for b, (ox, oy, oz) in enumerate(corners):
        y[b, oz:oz + 8, oy:oy + 16, ox:ox + 16] = rng.normal(size=(8, 16, 16))
    got = kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    for b, (ox, oy, oz) in enumerate(corners):
        want = oracle_adjoint_subvolume(g, op, y[b, oz:oz + 8, oy:oy + 16, ox:ox + 16], ox, oy, oz)
        check32(got[b], want, name=f"item {b} at {(ox, oy, oz)}")


def test_c3_dot_product_batch4(env, c3):
    torch, kats = env
    g, kp, op = c3
    rng = np.random.default_rng(33)
    xb = torch.from_numpy(rng.normal(size=(4,) + kp.sino_shape).astype(np.float32)).cuda()
    yb = torch.from_numpy(rng.normal(size=(4,) + kp.vol_shape).astype(np.float32)).cuda()
    ax = kp.recon(xb)
    aty = kp.adjoint(yb)
    for b in range(4):
        lhs = float((ax[b].double() * yb[b].double()).sum())
        rhs = float((xb[b].double() * aty[b].double()).sum())
        print(f"item {b}: <Ax,y> {lhs:.6e}, <x,A^T y> {rhs:.6e}")
        assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
