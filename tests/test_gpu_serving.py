"""Serving loop on the GPU: continuous batching of mixed geometries, sizes and
precisions.  Each result of a mixed, concurrent run must equal the same
request run alone (the same kernels on its own device block, so bit-equal),
and one is tied to the FP64 oracle.  Admission refusal, the wait limit, plan
eviction and an injected allocation failure are host-side failures: nothing
here faults or hangs the GPU."""
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


def mix_configs():
    """Small members of the serving mix: the config-1 scanner, and the clinical
    scanner (R 595, D 1085.6) with full, half and quarter column sets at
    several views per turn, pitch factors and volume sizes."""
    c1 = synth.config(1)
    clin = dict(R=595.0, D=1085.6, n_rows=64, n_cols_full=736, det_half_width=256.0, voxel=1.0)
    return [
        dict(c1),
        dict(clin, views_per_turn=580, turns=2, n_cols=368, col_keep=2, nx=64, ny=64, nz=16, pitch_factor=1.5),
        dict(clin, views_per_turn=256, turns=3, n_cols=736, col_keep=1, nx=96, ny=96, nz=24, pitch_factor=1.25),
        dict(clin, views_per_turn=290, turns=3, n_cols=184, col_keep=4, nx=48, ny=80, nz=20, pitch_factor=1.0),
    ]


def pinned_sino(torch, g, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(g["n_views"], g["n_rows"], g["n_cols"])).astype(np.float32)
    return torch.from_numpy(a).pin_memory()


def alone(kats, torch, g, sino, prec):
    plan = kats.Plan(g)
    vol = torch.empty((g["nz"], g["ny"], g["nx"]), dtype=torch.float32)
    plan.recon_host(sino, vol, precision=prec)
    return vol.numpy().copy()


def block_bytes(kats, g, prec):
    plan = kats.Plan(g)
    return kats.native.load().katsevich_host_workspace_bytes(plan.handle, 1, prec)


def test_mixed_stream_matches_each_request_alone(kats):
    import torch
    from paper_2201_02309_b300.serving import Server
    geoms = [kats.make_geometry(c) for c in mix_configs()]
    precs = [kats.KATS_PREC_FP32, kats.KATS_PREC_FP32, kats.KATS_PREC_FP16, kats.KATS_PREC_BF16]
    reqs = [(geoms[i % 4], precs[(i // 4 + i) % 4], 100 + i) for i in range(16)]
    biggest = max(block_bytes(kats, g, p) for g, p, _ in reqs)
    # room for about two of the largest blocks: requests queue, smaller ones backfill
    with Server(arena_bytes=int(2.5 * biggest), plan_cache_bytes=1 << 32, slots=3, max_bypass=4) as srv:
        sinos = [pinned_sino(torch, g, seed) for g, _, seed in reqs]  # all inputs ready: the requests arrive together
        tickets = [srv.submit(g, s, precision=p) for (g, p, _), s in zip(reqs, sinos)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_running"] >= 2, st  # work of several requests overlapped
    assert st["plan_misses"] == len(geoms) and st["plan_hits"] == len(reqs) - len(geoms)
    assert st["arena_peak_bytes"] <= int(2.5 * biggest)
    for (g, p, seed), (vol, rs) in zip(reqs, results):
        assert rs["status"] == 0 and rs["t_submit_ms"] <= rs["t_admit_ms"] <= rs["t_done_ms"]
        want = alone(kats, torch, g, pinned_sino(torch, g, seed), p)
        assert np.array_equal(vol.numpy(), want), (g["n_cols"], p)
    # one member tied to the oracle: the config-1 scanner in FP32
    g, p, seed = reqs[0]
    ref = oracle.Plan(g).recon(pinned_sino(torch, g, seed).numpy().astype(np.float64))
    check32(results[0][0].numpy(), ref)


def test_request_larger_than_arena_is_refused(kats):
    import torch
    from paper_2201_02309_b300.serving import Server
    g = kats.make_geometry(mix_configs()[0])
    with Server(arena_bytes=1 << 20, plan_cache_bytes=1 << 30, slots=2) as srv:
        t = srv.submit(g, pinned_sino(torch, g, 1))
        with pytest.raises(kats.KatsevichError) as e:
            srv.wait(t)
        assert e.value.status == kats.native.KATS_ENOMEM
        assert srv.stats()["refused"] == 1


def test_wait_limit_returns_timeout_and_keeps_ticket(kats):
    import torch
    from paper_2201_02309_b300.serving import Server
    g = kats.make_geometry(mix_configs()[2])
    with Server(arena_bytes=2 << 30, plan_cache_bytes=1 << 30, slots=2) as srv:
        t = srv.submit(g, pinned_sino(torch, g, 2))
        with pytest.raises(kats.KatsevichError) as e:
            srv.wait(t, timeout_ms=0)  # the plan alone takes longer than that
        assert e.value.status == kats.native.KATS_ETIMEOUT
        vol, rs = srv.wait(t)
        assert rs["status"] == 0
        assert np.array_equal(vol.numpy(), alone(kats, torch, g, pinned_sino(torch, g, 2), kats.KATS_PREC_FP32))


def test_plan_cache_evicts_idle_plans(kats):
    import torch
    from paper_2201_02309_b300.serving import Server
    geoms = [kats.make_geometry(c) for c in mix_configs()[:2]]
    order = [0, 1, 0, 1]
    with Server(arena_bytes=2 << 30, plan_cache_bytes=1, slots=2) as srv:
        for i, k in enumerate(order):
            vol, rs = srv.wait(srv.submit(geoms[k], pinned_sino(torch, geoms[k], 40 + i)))
            assert rs["plan_hit"] == 0
            assert np.array_equal(vol.numpy(), alone(kats, torch, geoms[k], pinned_sino(torch, geoms[k], 40 + i),
                                                      kats.KATS_PREC_FP32))
        st = srv.stats()
    assert st["plan_misses"] == 4 and st["plan_evictions"] >= 3 and st["plans_cached"] <= 1


def test_injected_allocation_failures(kats):
    import torch
    from paper_2201_02309_b300.serving import Server
    native = kats.native
    native.katsevich_debug_fail_allocs(1)
    with pytest.raises(kats.KatsevichError) as e:
        Server(arena_bytes=1 << 28, plan_cache_bytes=1 << 30, slots=2)
    assert e.value.status == native.KATS_ENOMEM
    g = kats.make_geometry(mix_configs()[3])
    with Server(arena_bytes=1 << 30, plan_cache_bytes=1 << 30, slots=2) as srv:
        native.katsevich_debug_fail_allocs(1)  # the next plan build fails
        t = srv.submit(g, pinned_sino(torch, g, 9))
        with pytest.raises(kats.KatsevichError) as e:
            srv.wait(t)
        assert e.value.status == native.KATS_ENOMEM
        vol, rs = srv.wait(srv.submit(g, pinned_sino(torch, g, 9)))  # recovers: the plan builds now
        assert rs["status"] == 0
        assert np.array_equal(vol.numpy(), alone(kats, torch, g, pinned_sino(torch, g, 9), kats.KATS_PREC_FP32))
    native.katsevich_debug_fail_allocs(0)


def test_large_requests_take_the_overlapped_path_in_the_mix(kats):
    """Requests whose view window is 128 MiB or more run the overlapped host path
    (chunked copies, filter stream, chunk-by-chunk first slab) inside the server,
    concurrently with small ones; each result equals the same request run alone."""
    import torch
    from paper_2201_02309_b300.serving import Server
    big = dict(synth.config(2))
    big.update(nx=64, ny=64, nz=48)
    gb = kats.make_geometry(big)
    pb = kats.Plan(gb)
    assert (pb.info["n_filtered_views"] + 1) * gb["n_rows"] * gb["n_cols"] * 4 >= (128 << 20)
    gs = kats.make_geometry(mix_configs()[1])
    reqs = [(gb, kats.KATS_PREC_FP32, 201), (gs, kats.KATS_PREC_FP32, 202), (gb, kats.KATS_PREC_FP16, 203),
            (gs, kats.KATS_PREC_BF16, 204)]
    with Server(arena_bytes=4 * block_bytes(kats, gb, kats.KATS_PREC_FP32), plan_cache_bytes=1 << 32, slots=3,
                max_bypass=4) as srv:
        sinos = [pinned_sino(torch, g, seed) for g, _, seed in reqs]
        tickets = [srv.submit(g, s, precision=p) for (g, p, _), s in zip(reqs, sinos)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["max_running"] >= 2, st
    for (g, p, seed), (vol, rs) in zip(reqs, results):
        assert rs["status"] == 0
        assert np.array_equal(vol.numpy(), alone(kats, torch, g, pinned_sino(torch, g, seed), p)), (g["nx"], p)
