"""Full-size parity: the 512 x 512 x 256 clinical workload (64 x 736 detector,
1160 views/turn, 8 turns) reconstructed on the GPU in the benchmark's launch
configuration, checked against the FP64 oracle on sampled voxels (PI windows
from the oracle's own PI-line solver, filtered views from the oracle's
filter on exactly the views those voxels need) and on sampled filtered views.
"""
import numpy as np
import pytest

import oracle
import synth
from cases import check32, close_paths, near_tie, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def c2():
    import torch

    import paper_2201_02309_b300 as kats
    cfg = synth.config(2)
    g = oracle.derive_geometry(cfg)
    ell = synth.phantom_for(cfg, g, synth.phantom_seed(2))
    sino = synth.project(g, ell).astype(np.float32)
    kp = kats.Plan(g)
    dsino = torch.from_numpy(sino).cuda()
    vol = kp.recon(dsino)
    torch.cuda.synchronize()
    return g, sino, kp, dsino, vol.cpu().numpy()


def test_c2_plan_info_and_slabs(c2):
    g, sino, kp, _, _ = c2
    info = kp.info
    assert info["slices_per_pitch"] == 70 and g["P"] == 70.0
    # sampled columns of the one-pitch table vs the oracle's PI solver
    rng = np.random.default_rng(0)
    ijk = np.stack([rng.integers(0, 512, 3000), rng.integers(0, 512, 3000), rng.integers(0, 70, 3000)], 1)
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    k0, k1, w0, w1 = kp.table("k0"), kp.table("k1"), kp.table("w0"), kp.table("w1")
    i, j, s = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    bad0 = (k0[s, j, i] != ka) & ~near_tie(wa)
    bad1 = (k1[s, j, i] != kb) & ~near_tie(wb)
    assert not bad0.any() and not bad1.any()
    ok = k0[s, j, i] == ka
    assert np.abs(w0[s, j, i] - wa)[ok].max() < 2e-7


def test_c2_filtered_views_sampled(c2):
    import torch
    g, sino, kp, dsino, _ = c2
    gF = kp.filter(dsino)
    torch.cuda.synchronize()
    op = oracle.Plan(g, with_pi=False)
    v0 = kp.info["first_view"]
    for v in (0, 1777, kp.info["n_filtered_views"] - 1):
        want = op.filter(sino.astype(np.float64), v0 + v, 1)[0]
        check32(gF[v, :, :g["n_cols"]].cpu().numpy(), want)


def test_c2_voxels_sampled(c2):
    g, sino, kp, _, vol = c2
    rng = np.random.default_rng(1)
    n = 240
    s = rng.integers(127, 130, n)
    ijk = np.stack([rng.integers(0, 512, n), rng.integers(0, 512, n), s], 1)
    # ragged corners and the volume edges of those slices
    ijk[:4, :2] = [(0, 0), (511, 0), (0, 511), (511, 511)]
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    v0, v1 = int(ka.min()), int(kb.max())
    op = oracle.Plan(g, with_pi=False)
    gF = op.filter(sino.astype(np.float64), v0, v1 - v0 + 1)
    want = oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb))
    got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    check32(got, want)
    assert np.isfinite(vol).all()
    assert kp.info["update_count"] > 4.0e10
    import paper_2201_02309_b300 as kats
    assert kats.native.katsevich_device_status(kp.handle) == 0


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_c2_host_pipeline_matches_device(c2, prec):
    """katsevich_recon_host at full size (overlapped window chunks, volume slabs) gives the
    device-buffer result of katsevich_recon: to FP32 rounding, since its middle slab pairs
    slices one pitch apart within the slab while the whole-volume launch pairs them from
    slice 0."""
    import torch

    import paper_2201_02309_b300 as kats
    g, sino, kp, dsino, vol = c2
    p = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16}[prec]
    dev = vol if prec == "fp32" else kp.recon(dsino, precision=p).cpu().numpy()
    hs = torch.from_numpy(sino).pin_memory()
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(hs, hv, precision=p)
    if prec == "fp32":
        close_paths(hv.numpy(), dev, "host pipeline")
    else:  # 16-bit storage rounds the filtered data: the two groupings agree to that rounding
        assert rel_l2(hv.numpy(), dev) < 1e-4
    assert np.isfinite(hv.numpy()).all()


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_host_pipeline_small_volume_long_window(prec):
    """The overlapped host path on a 64 x 64 x 48 volume of the clinical scanner:
    its view window (about 1300 views of 64 x 736, above the pipeline's 128 MiB
    threshold) arrives in chunks, the first 16-slice slab is backprojected chunk
    by chunk from raw partial sums, and the result equals the device-buffer
    reconstruction bit for bit."""
    import torch

    import paper_2201_02309_b300 as kats
    cfg = dict(synth.config(2))
    cfg.update(nx=64, ny=64, nz=48)
    g = kats.make_geometry(cfg)
    kp = kats.Plan(g)
    nf = kp.info["n_filtered_views"]
    assert (nf + 1) * g["n_rows"] * g["n_cols"] * 4 >= (128 << 20)
    p = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16, "bf16": kats.KATS_PREC_BF16}[prec]
    rng = np.random.default_rng(5)
    sino = rng.standard_normal(kp.sino_shape).astype(np.float32)
    dev = kp.recon(torch.from_numpy(sino).cuda(), precision=p).cpu().numpy()
    hs = torch.from_numpy(sino).pin_memory()
    hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
    kp.recon_host(hs, hv, precision=p)
    assert np.array_equal(hv.numpy(), dev)
    assert np.isfinite(dev).all() and np.abs(dev).max() > 0


def compare_int_table(got, want, want_frac, name):
    """Integer table bit for bit; a mismatch is allowed only at a floor tie (the oracle's
    fraction within 1e-9 of an integer).  Returns (mismatches, ties seen)."""
    bad = got != want
    ties = near_tie(want_frac)
    assert not (bad & ~ties).any(), f"{name}: {int((bad & ~ties).sum())} mismatches away from ties"
    print(f"{name}: {int(bad.sum())} mismatches, {int(ties.sum())} near-ties of {got.size}")
    return int(bad.sum()), int(ties.sum())


def compare_kappa_psi(kp, op):
    # the backward-rebinning root psi_hat with the smallest |psi| (Sec. II, Eq. (w_k)): the
    # device's safeguarded Newton against the oracle's bisection, on every detector sample
    compare_int_table(kp.table("kappa_idx"), op.kap[0], op.kap[1], "kappa_idx")
    same = kp.table("kappa_idx") == op.kap[0]
    assert np.abs(kp.table("kappa_frac") - op.kap[1])[same].max() < 2e-7
    compare_int_table(kp.table("psi_idx"), op.psi[0], op.psi[1], "psi_idx")
    same = kp.table("psi_idx") == op.psi[0]
    assert np.abs(kp.table("psi_frac") - op.psi[1])[same].max() < 2e-7


def test_c2_kappa_psi_tables_clinical_fan(c2):
    """The clinical fan (alpha_m = 0.654), where w_kappa turns over in psi and the
    smallest-|psi| rule picks the root."""
    g, _, kp, _, _ = c2
    op = oracle.Plan(g, with_pi=False)
    assert oracle.alpha_m(g) > 0.65
    assert kp.table("psi_idx").shape == (64, 736) and kp.table("kappa_idx").shape == (128, 735)
    compare_kappa_psi(kp, op)
    # the smallest-root rule is exercised: detector samples whose w also has a second root
    # further out on the same branch (past the turnover of w_kappa in psi)
    assert second_root_samples(g, op) > 500


def second_root_samples(g, op):
    pm = 0.5 * np.pi + oracle.alpha_m(g)
    idx, frac = op.psi
    psi = -pm + (idx + frac) * (2 * pm / (oracle.n_psi(g) - 1))
    nr, nc = idx.shape
    alpha = (np.arange(nc) - 0.5 * (nc - 1)) * g["d_alpha"] + g["alpha_offset"]
    w = (np.arange(nr) - 0.5 * (nr - 1)) * g["d_w"] + g["w_offset"]
    n = 0
    for c in range(nc):
        end_hi, end_lo = oracle.w_kappa(g, alpha[c], pm), oracle.w_kappa(g, alpha[c], -pm)
        for r in range(nr):
            if idx[r, c] < 0:
                continue
            n += alpha[c] > 0 and psi[r, c] > 0 and w[r] >= end_hi
            n += alpha[c] < 0 and psi[r, c] < 0 and w[r] <= end_lo
    print(f"samples with a second, larger root: {n}")
    return n


SLICES_C2 = [0, 15, 16, 69, 70, 71, 139, 140, 255]


def test_c2_pi_table_across_pitch_boundaries(c2):
    """Slices on both sides of each pitch boundary read table slice s mod 70 with their
    views shifted by (s div 70) turns: checked against the oracle's own PI solver for the
    voxel itself (no table)."""
    g, _, kp, _, _ = c2
    rng = np.random.default_rng(11)
    cols = [(0, 0), (511, 0), (0, 511), (511, 511), (15, 16), (16, 15), (255, 256), (256, 255)]
    ijk = []
    for s in SLICES_C2:
        ijk += [(i, j, s) for i, j in cols]
        ijk += [(int(i), int(j), s) for i, j in rng.integers(0, 512, (60, 2))]
    ijk = np.array(ijk)
    ka, kb, wa, wb = oracle.pi_windows(g, ijk)
    N, vpt = 70, g["views_per_turn"]
    k0, k1, w0, w1 = kp.table("k0"), kp.table("k1"), kp.table("w0"), kp.table("w1")
    i, j, s = ijk[:, 0], ijk[:, 1], ijk[:, 2]
    gk0 = k0[s % N, j, i] + (s // N) * vpt
    gk1 = k1[s % N, j, i] + (s // N) * vpt
    assert not ((gk0 != ka) & ~near_tie(wa)).any() and not ((gk1 != kb) & ~near_tie(wb)).any()
    ok = (gk0 == ka) & (gk1 == kb)
    assert np.abs(w0[s % N, j, i] - wa)[ok].max() < 2e-7 and np.abs(w1[s % N, j, i] - wb)[ok].max() < 2e-7


def test_c2_voxels_boundary_slices(c2):
    """Sampled voxels in the first and last 16-slice tiles, on both sides of the pitch
    boundaries (69/70/71, 139/140) and of a 16 x 16 tile boundary, and the four corner
    columns (the ones whose views take the longest ramps), against the oracle's chain on
    exactly the views each group of slices needs."""
    g, sino, kp, _, vol = c2
    rng = np.random.default_rng(12)
    op = oracle.Plan(g, with_pi=False)
    cols = [(0, 0), (511, 0), (0, 511), (511, 511), (15, 15), (16, 16), (15, 16), (16, 15), (255, 256)]
    got_all, want_all = [], []
    for group in ([0, 15, 16], [69, 70, 71], [139, 140], [255]):
        ijk = []
        for s in group:
            ijk += [(i, j, s) for i, j in cols]
            ijk += [(int(i), int(j), s) for i, j in rng.integers(0, 512, (40, 2))]
        ijk = np.array(ijk)
        ka, kb, wa, wb = oracle.pi_windows(g, ijk)
        v0, v1 = int(ka.min()), int(kb.max())
        gF = op.filter(sino.astype(np.float64), v0, v1 - v0 + 1)
        want_all.append(oracle.backproject_points(g, gF, v0, ijk, (ka, kb, wa, wb)))
        got_all.append(vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]])
        check32(got_all[-1], want_all[-1], name=f"slices {group}")
    check32(np.concatenate(got_all), np.concatenate(want_all), name="all boundary samples")
