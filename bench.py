#!/usr/bin/env python
"""Benchmark of the Katsevich helical cone-beam reconstruction operator.

One step = one full reconstruction (steps 1-7 of the paper's Section II) of
the clinical workload: 512 x 512 x 256 volume at 1 mm, curved detector
64 x 736, 1160 views/turn, 8 turns, maximal-fit pitch (70 mm), seeded random
ellipsoid phantom (FP64 line integrals, stored FP32).  The metric is GUPS:
voxel-view updates (each voxel's PI-window view count, summed) per second.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank reconstructs its own volume (independent
problems, no collective on the data path: weak scaling) and rank 0 prints one
JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Katsevich recon GUPS (voxel·views/s), vol/s, p50/p99 latency vs plain FP32"
UNIT = "GUPS (1e9 voxel-view updates/s)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp16"], default="fp32",
                    help="storage precision of the intermediate data (precision form)")
    ap.add_argument("--shard", choices=["replicas", "slabs"], default="replicas",
                    help="N > 1: one volume per rank (weak scaling) or one volume split into z-slabs (strong)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="config 2: leave the precision, differentiation and serving forms out of the JSON line")
    ap.add_argument("--nz", type=int, default=None, help="smaller volume height (profiling captures only)")
    ap.add_argument("--turns", type=int, default=None, help="fewer helix turns (profiling captures only)")
    ap.add_argument("--simulate", action="store_true", help="time the data-simulation pipeline instead")
    ap.add_argument("--requests", type=int, default=256, help="config 5: requests in the stream")
    ap.add_argument("--slots", type=int, default=4, help="config 5: concurrent requests (CUDA streams)")
    ap.add_argument("--arena-gb", type=float, default=24.0, help="config 5: device arena for running requests")
    ap.add_argument("--plan-cache-gb", type=float, default=16.0, help="config 5: device plan cache")
    return ap.parse_args()


def config_for(args):
    import synth
    cfg = synth.config(args.config)
    if args.nz:
        cfg["nz"] = args.nz
        cfg["name"] += f"_nz{args.nz}"
    if args.turns:
        cfg["turns"] = args.turns
        cfg["name"] += f"_turns{args.turns}"
    return cfg


def captured_traffic(kernel):
    """DRAM bytes per launch from the committed ncu capture, or None once the
    kernel's source differs from the one that capture measured."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha1()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, KeyError, ValueError):
        return None
    return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["source_sha1"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(cfg_index, geom, cfg):
    import numpy as np

    import synth
    ell = synth.phantom_for(cfg, geom, synth.phantom_seed(cfg_index))
    sino = synth.project(geom, ell)
    sino = synth.add_noise(sino, cfg["noise_sigma"], synth.noise_seed(cfg_index))
    return cfg, sino.astype(np.float32)


def describe(cfg, g, info, world=1, slabs=False):
    """The workload (identical on both arms of the benchmark; the arithmetic type is the line's dtype)."""
    return {"workload": cfg["name"], "volume_xyz": [g["nx"], g["ny"], g["nz"]], "voxel_mm": g["dx"],
            "detector_rows_cols": [g["n_rows"], g["n_cols"]], "views": g["n_views"],
            "views_per_turn": g["views_per_turn"], "pitch_mm": g["P"], "R_mm": g["R"], "D_mm": g["D"],
            "slices_per_pitch": info["slices_per_pitch"], "n_psi": info["n_psi"],
            "filtered_views": info["n_filtered_views"], "updates_per_volume": info["update_count"],
            "batch_per_gpu": 1, "parallelism": f"z-slabs x{world}" if slabs else f"replicas x{world}",
            "l2": "inputs larger than L2 (sinogram %.2f GB, filtered view window %.2f GB)" % (
                g["n_views"] * g["n_rows"] * g["n_cols"] * 4 / 1e9,
                info["n_filtered_views"] * g["n_rows"] * g["n_cols"] * 4 / 1e9)}


# --------------------------------------------------------------------------- oracle
def oracle_sample(g, sino, info, n_filter_views=128):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload and
    extrapolate to one full reconstruction: the backprojection of one whole slice
    (every voxel of slice nz/2 over its own PI window) and the filter (steps 1-6) on
    n_filter_views of the views that slice reads; filter time per view x filtered
    views + backprojection time per update x update count.  The filter does the same
    work for every view, so a block of views stands for all of them."""
    import numpy as np

    import oracle
    op = oracle.Plan(g, with_pi=False)
    s = g["nz"] // 2
    ii, jj = np.meshgrid(np.arange(g["nx"]), np.arange(g["ny"]), indexing="xy")
    ijk = np.stack([ii.ravel(), jj.ravel(), np.full(ii.size, s)], 1)
    win = oracle.pi_windows(g, ijk)
    a, b = int(win[0].min()), int(win[1].max())
    nf = min(n_filter_views, b - a + 1)
    v0 = (a + b - nf) // 2  # a block of views from the middle of the slice's window
    t = time.perf_counter()
    gF_part = op.filter(sino, v0, nf)
    t_filter = time.perf_counter() - t
    gF = np.zeros((b - a + 1, g["n_rows"], g["n_cols"]))
    gF[v0 - a:v0 - a + nf] = gF_part
    t = time.perf_counter()
    oracle.backproject_points(g, gF, a, ijk, win)
    t_bp = time.perf_counter() - t
    upd = int((win[1] - win[0] + 1).sum())
    est = t_filter / nf * info["n_filtered_views"] + t_bp / upd * info["update_count"]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": info["update_count"] / est / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle (C, OpenMP, {cores} threads): backprojection of all {ijk.shape[0]} voxels of "
                      f"slice {s} over their PI windows ({upd} updates, {t_bp:.1f} s) and the filter on {nf} of "
                      f"the {b - a + 1} views that slice reads ({t_filter:.1f} s), extrapolated linearly in "
                      f"updates and filtered views to one full volume ({est:.0f} s)",
            "seconds": t_filter + t_bp}


def oracle_patch(g, sino, s, x0, y0, n=16):
    """The oracle's values of an n x n patch of slice s (every view those voxels read
    filtered by the oracle): the reference the reduced-precision forms are measured
    against at full size.  Returns (ijk, values)."""
    import numpy as np

    import oracle
    ii, jj = np.meshgrid(np.arange(x0, x0 + n), np.arange(y0, y0 + n), indexing="xy")
    ijk = np.stack([ii.ravel(), jj.ravel(), np.full(ii.size, s)], 1)
    win = oracle.pi_windows(g, ijk)
    a, b = int(win[0].min()), int(win[1].max())
    gF = oracle.Plan(g, with_pi=False).filter(sino, a, b - a + 1)
    return ijk, oracle.backproject_points(g, gF, a, ijk, win)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    cfg = config_for(args)
    g = oracle.derive_geometry(cfg)
    # the oracle's own one-pitch table gives the update count and the filtered view window
    t = oracle.pi_table(g)
    N = oracle.pitch_slices(g)
    s = list(range(g["nz"]))
    upd = sum(int((t["k1"][j] - t["k0"][j] + 1).sum()) for j in (x % N for x in s))
    kmin = min(int(t["k0"][x % N].min()) + (x // N) * g["views_per_turn"] for x in s)
    kmax = max(int(t["k1"][x % N].max()) + (x // N) * g["views_per_turn"] for x in s)
    info = {"first_view": kmin, "n_filtered_views": kmax - kmin + 1, "update_count": upd,
            "slices_per_pitch": N, "n_psi": oracle.n_psi(g), "workspace_bytes": 0}
    _, sino = workload(args.config, g, cfg)
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(g, sino, info)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median(x["value"] for x in vals)
    secs = sum(x["seconds"] for x in vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(cfg, g, info, args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- ours
def job_throughput(ms_local, updates_per_rank, world, max_over_ranks):
    """Whole-job GUPS: every rank's updates over the slowest rank's time."""
    ms = max_over_ranks(ms_local)
    return ms, updates_per_rank * world / (ms / 1e3) / 1e9


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2201_02309_b300 as kats
    from paper_2201_02309_b300 import build as kbuild
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    kbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cfg = config_for(args)
    g = kats.make_geometry(cfg)
    cfg, sino_np = workload(args.config, g, cfg)
    plan = kats.Plan(g)
    info = plan.info
    prec = {"fp32": kats.KATS_PREC_FP32, "bf16": kats.KATS_PREC_BF16, "fp16": kats.KATS_PREC_FP16}[args.precision]
    slabs = args.shard == "slabs"
    sino = torch.from_numpy(sino_np).to(dev)
    vol = torch.empty(plan.vol_shape, dtype=torch.float32, device=dev)
    ws = plan.workspace(precision=prec, device=dev)
    stream = torch.cuda.current_stream(dev)
    if slabs:
        # this rank's slices of the one volume and just the sinogram views they read
        s0, s1 = kats.slab_partition(g["nz"], world)[rank]
        vb, vc = plan.slab_views(s0, s1) if s1 > s0 else (0, 0)
        win = sino[vb:vb + vc].clone()
        vol_slab = torch.empty((s1 - s0, g["ny"], g["nx"]), dtype=torch.float32, device=dev)
        del sino

    def step():
        if not slabs:
            plan.recon(sino, out=vol, workspace=ws, precision=prec)
        elif s1 > s0:
            plan.recon_slab(win, vb, s0, s1, out=vol_slab, workspace=ws, precision=prec)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x, op=None):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=op or dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = kats.native.katsevich_launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    launches = kats.native.katsevich_launch_count() - n_launch0  # the library's own count
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    volumes = 1 if slabs else world  # volumes the whole job reconstructs per step
    ms, value = job_throughput(e0.elapsed_time(e1) / args.steps, info["update_count"], volumes, max_over_ranks)
    updates = info["update_count"] * volumes

    roofline = None
    if args.precision == "fp32" and not slabs:
        # per-kernel durations over the same work (events on the launching stream)
        gF = torch.empty(plan.filtered_shape, dtype=torch.float32, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            ev[3 * i].record(stream)
            kats.native.katsevich_filter(plan.handle, sino.data_ptr(), gF.data_ptr(), 1, 0, ws.data_ptr(), ws.numel(),
                                         stream.cuda_stream)
            ev[3 * i + 1].record(stream)
            kats.native.katsevich_backproject(plan.handle, gF.data_ptr(), vol.data_ptr(), 1, stream.cuda_stream)
            ev[3 * i + 2].record(stream)
        torch.cuda.synchronize()
        t_filter = statistics.mean(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(args.steps))
        t_bp = statistics.mean(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(args.steps))

        pk, pk_kind = peaks()
        sm_mhz = float(pk.get("sm_max_mhz", 2032.0))
        # Backprojection reads 4 fp32 detector taps (16 B) per voxel-view update from the
        # shared-memory window the TMA stages; its roofline is the SM data path
        # (148 SMs x 128 B/clk x clock), not HBM.
        bytes_per_update = 16.0
        smem_peak = 148 * 128 * sm_mhz * 1e6 / 1e9  # GB/s
        alg_bytes = info["update_count"] * bytes_per_update
        achieved = alg_bytes / (t_bp / 1e3) / 1e9
        # the same path's read bandwidth measured on this GPU (conflict-free 16-byte shared loads), and
        # the hardware bilinear texture-fetch rate a texture-based gather would be bound by
        smem_measured = kats.native.katsevich_smem_read_bandwidth() / 1e9
        tex32 = kats.native.katsevich_tex_bilinear_rate(False)
        tex16 = kats.native.katsevich_tex_bilinear_rate(True)
        updates_per_s = info["update_count"] / (t_bp / 1e3)
        roofline = {"kernel": "backprojection (k_backproject_multi + k_backproject_tma, one reconstruction's launches)",
                    "bound": "alu", "achieved": achieved, "peak": smem_peak,
                    "unit": "GB/s", "frac": achieved / smem_peak, "traffic": captured_traffic("backprojection"),
                    "peak_source": f"shared-memory data path: 148 SMs x 128 B/clk x {sm_mhz:.0f} MHz ({pk_kind} clock)",
                    "peak_measured": smem_measured, "frac_of_measured": achieved / smem_measured,
                    "tex_bilinear_gsamples_per_s": {"fp32": tex32 / 1e9, "fp16": tex16 / 1e9},
                    "updates_over_tex_fp32": updates_per_s / tex32,
                    "algorithmic_bytes_per_launch": alg_bytes, "ms_per_launch": t_bp, "filter_ms": t_filter}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e and slabs:
        # the slab's views from pinned host memory, the slab back: sequential copies around recon_slab
        hs = torch.from_numpy(sino_np[vb:vb + vc]).pin_memory()
        hv = torch.empty(tuple(vol_slab.shape), dtype=torch.float32).pin_memory()

        def host_step():
            win.copy_(hs, non_blocking=True)
            step()
            hv.copy_(vol_slab, non_blocking=True)
            torch.cuda.synchronize()
        for _ in range(max(1, args.warmup)):
            host_step()
        barrier()
        times = []
        for _ in range(args.steps):
            t = time.perf_counter()
            host_step()
            times.append(time.perf_counter() - t)
        te = max_over_ranks(statistics.mean(times))
        # bytes of the whole job: every rank's copies
        h2d = max_over_ranks(float(hs.numel() * 4), dist.ReduceOp.SUM)
        d2h = max_over_ranks(float(hv.numel() * 4), dist.ReduceOp.SUM)
        e2e = {"value": updates / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": te * 1e3}
    elif not args.no_e2e:
        hs = torch.from_numpy(sino_np).pin_memory()
        hv = torch.empty(plan.vol_shape, dtype=torch.float32).pin_memory()
        wsh = torch.empty(kats.native.katsevich_host_workspace_bytes(plan.handle, 1, prec), dtype=torch.uint8,
                          device=dev)
        for _ in range(max(1, args.warmup)):
            plan.recon_host(hs, hv, workspace=wsh, precision=prec)
        barrier()
        times = []
        for _ in range(args.steps):
            t = time.perf_counter()
            plan.recon_host(hs, hv, workspace=wsh, precision=prec)
            times.append(time.perf_counter() - t)
        te = max_over_ranks(statistics.mean(times))
        h2d = (info["n_filtered_views"] + 1) * g["n_rows"] * g["n_cols"] * 4
        e2e = {"value": updates / te / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(np.prod(plan.vol_shape)) * 4, "ms_per_step": te * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not slabs:
        # the host is shared: the median of three runs of the sample
        runs = sorted((oracle_sample(g, sino_np, info) for _ in range(3)), key=lambda r: r["value"])
        cpu = runs[1]
        cpu.pop("seconds", None)
        cpu["sample"] += "; median of 3 runs (%.3f / %.3f / %.3f GUPS)" % tuple(r["value"] for r in runs)

    forms = None
    if rank == 0 and world == 1 and not slabs and not args.no_forms and args.precision == "fp32" and \
            args.config == 2 and not args.nz and not args.turns:
        forms = other_forms(args, plan, g, sino, sino_np, vol, ws, ms)

    if rank == 0:
        config = describe(cfg, g, info, world, slabs)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong" if slabs else "weak",
                "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[args.precision],
                "data": "synthetic", "config": config, "vol_per_s": volumes / (ms / 1e3),
                "workspace_bytes": info["workspace_bytes"],
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        if forms is not None:
            line.update(forms)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------- other forms
def other_forms(args, plan, g, sino, sino_np, vol32, ws32, ms32):
    """The three other forms of the operator, measured in the same run as the FP32 line:
    BF16 / FP16 storage on the same workload (device step, GUPS, ratio to the FP32 step, and
    accuracy against the FP64 oracle on a 16 x 16 voxel patch of the middle slice: rel-L2 and
    max-abs, beside the FP32 path's own); config 3 forward + backward of the differentiable layer
    (batch 4); the serving mix saturated and at rho = 0.8, with served over plain FP32."""
    import numpy as np
    import torch

    import paper_2201_02309_b300 as kats
    dev = sino.device
    stream = torch.cuda.current_stream(dev)
    upd = plan.info["update_count"]
    s, x0, y0 = g["nz"] // 2, 3 * g["nx"] // 8, g["ny"] // 4
    ijk, want = oracle_patch(g, sino_np, s, x0, y0)

    def accuracy(v):
        got = v[ijk[:, 2], ijk[:, 1], ijk[:, 0]].astype(np.float64)
        return {"rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                "max_abs": float(np.abs(got - want).max()), "max_abs_over_max": float(
                    np.abs(got - want).max() / np.abs(want).max())}

    prec_out = {"oracle_sample": f"16 x 16 voxels of slice {s} at x, y >= ({x0}, {y0}), every view they read "
                                 "filtered by the FP64 oracle",
                "fp32": dict(ms_per_step=ms32, gups=upd / ms32 * 1e-6, **accuracy(vol32.cpu().numpy()))}
    for name, p in (("fp16", kats.KATS_PREC_FP16), ("bf16", kats.KATS_PREC_BF16)):
        ws = plan.workspace(precision=p, device=dev)
        out = torch.empty(plan.vol_shape, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            plan.recon(sino, out=out, workspace=ws, precision=p)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.recon(sino, out=out, workspace=ws, precision=p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        prec_out[name] = dict(ms_per_step=ms, gups=upd / ms * 1e-6, over_fp32=ms32 / ms,
                              **accuracy(out.cpu().numpy()))
        del out
    diff = differentiation_result(argparse.Namespace(steps=max(3, args.steps // 2), warmup=2))
    srv = serving_result(argparse.Namespace(requests=args.requests, slots=args.slots, arena_gb=args.arena_gb,
                                            plan_cache_gb=args.plan_cache_gb, precision="fp32"), rhos=(0.8,))
    sv = srv["serving"]
    return {"precision_forms": prec_out,
            "differentiation": {"workload": diff["config"]["workload"], "batch": diff["config"]["batch"],
                                "forward_ms": diff["forward_ms"], "backward_ms": diff["backward_ms"],
                                "ms_per_batch": diff["ms_per_step"], "gups_fwd_bwd": diff["value"],
                                "gpu_launches": diff["gpu_launches"]},
            "serving": {"workload": srv["config"]["workload"], "requests": srv["config"]["requests"],
                        "slots": srv["config"]["slots"], "saturated": sv["saturated"],
                        "rho_0.8": sv["poisson"]["0.8"], "plain_fp32_vol_per_s": sv["plain_fp32"]["vol_per_s"],
                        "served_over_plain": sv["served_over_plain"],
                        "gpu_launches": srv["gpu_launches"]}}


# ----------------------------------------------------------------- serving form
SERVING_VOLUMES = [(128, 128, 32), (256, 256, 64), (512, 512, 128)]
SERVING_VPT = [256, 580, 1160]
SERVING_DETECTORS = [(736, 1), (368, 2), (184, 4)]  # columns kept, every col_keep-th of the 736
SERVING_PITCH = [1.0, 1.25, 1.5]


def serving_protocols(kats, n_protocols=12, seed=7):
    """Scan protocols of the serving mix, drawn (seeded) from the product of the
    volume sizes, views per turn, detector column sets and pitch factors; the
    clinical scanner (R 595, D 1085.6, 64 rows).  Turns: the volume's pitches
    plus two, so every PI window lies inside the scan."""
    import math

    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_protocols):
        (nx, ny, nz) = SERVING_VOLUMES[rng.integers(3)]
        vpt = SERVING_VPT[rng.integers(3)]
        cols, keep = SERVING_DETECTORS[rng.integers(3)]
        pf = SERVING_PITCH[rng.integers(3)]
        cfg = dict(R=595.0, D=1085.6, views_per_turn=vpt, turns=1, n_rows=64, n_cols=cols, n_cols_full=736,
                   col_keep=keep, det_half_width=256.0, nx=nx, ny=ny, nz=nz, voxel=1.0, pitch_factor=pf)
        g = kats.make_geometry(cfg)
        cfg["turns"] = int(math.ceil(nz * g["dz"] / g["P"])) + 2
        out.append(kats.make_geometry(cfg))
    return out


def run_serving(args):
    print(json.dumps(serving_result(args)))


def serving_result(args, rhos=(0.5, 0.8, 1.0)):
    """Config 5: a seeded Poisson stream of requests over mixed protocols,
    served with continuous batching; p50/p99 latency and vol/s, next to the
    plain FP32 path (one request at a time through katsevich_recon_host)."""
    import collections

    import numpy as np
    import torch

    import paper_2201_02309_b300 as kats
    from paper_2201_02309_b300 import build, native
    from paper_2201_02309_b300.serving import Server
    build.build()
    n_req, slots, seed = args.requests, args.slots, 7
    prec = {"fp32": kats.KATS_PREC_FP32, "bf16": kats.KATS_PREC_BF16, "fp16": kats.KATS_PREC_FP16}[args.precision]
    protos = serving_protocols(kats)
    rng = np.random.default_rng(seed)
    which = rng.integers(len(protos), size=n_req)
    plans = [kats.Plan(g) for g in protos]
    updates = [p.info["update_count"] for p in plans]
    gen = torch.Generator(device="cuda").manual_seed(seed)
    sinos = []
    for g in protos:
        s = torch.empty((g["n_views"], g["n_rows"], g["n_cols"]), dtype=torch.float32, pin_memory=True)
        s.copy_(torch.rand(s.shape, generator=gen, device="cuda"))
        sinos.append(s)
    max_vol = max(g["nx"] * g["ny"] * g["nz"] for g in protos)
    depth = 3 * slots
    pool = [torch.empty(max_vol, dtype=torch.float32, pin_memory=True) for _ in range(depth)]

    def vol_view(buf, g):
        return buf[: g["nz"] * g["ny"] * g["nx"]].view(g["nz"], g["ny"], g["nx"])

    # plain FP32 path: one request at a time, synchronous, plans built beforehand
    ws = torch.empty(max(native.load().katsevich_host_workspace_bytes(p.handle, 1, kats.KATS_PREC_FP32)
                         for p in plans), dtype=torch.uint8, device="cuda")
    for k in range(len(protos)):  # warm-up
        plans[k].recon_host(sinos[k], vol_view(pool[0], protos[k]), workspace=ws)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in which:
        plans[int(k)].recon_host(sinos[k], vol_view(pool[0], protos[k]), workspace=ws)
    plain_s = time.perf_counter() - t
    mu = n_req / plain_s  # single-stream capacity, requests/s
    del ws
    torch.cuda.empty_cache()

    arena = int(args.arena_gb * (1 << 30))

    def serve(arrivals, closed_loop):
        """Submit request i at arrivals[i] (seconds; closed loop: as soon as fewer
        than `depth` are outstanding).  Returns latencies (ms), makespan (s), stats."""
        lat, free, out = [None] * n_req, list(range(depth)), collections.deque()
        first_submit, last_done = None, 0.0
        with Server(arena_bytes=arena, plan_cache_bytes=int(args.plan_cache_gb * (1 << 30)), slots=slots,
                    max_bypass=2 * slots) as srv:
            for k in range(len(protos)):  # plans cached on the device before the stream starts
                srv.wait(srv.submit(protos[k], sinos[k], vol_view(pool[0], protos[k]), precision=prec))
            t0 = time.perf_counter()
            n_launch0 = native.katsevich_launch_count()
            i = 0
            while i < n_req or out:
                now = time.perf_counter() - t0
                if i < n_req and free and (closed_loop or now >= arrivals[i]):
                    k, b = int(which[i]), free.pop()
                    tk = srv.submit(protos[k], sinos[k], vol_view(pool[b], protos[k]), precision=prec)
                    late = 0.0 if closed_loop else (time.perf_counter() - t0) - arrivals[i]
                    out.append((i, tk, b, late))
                    i += 1
                    continue
                if out:
                    j, tk, b, late = out[0]
                    rc, st, msg = native.katsevich_server_wait(srv.handle, tk.id, 0)
                    if rc == native.KATS_ETIMEOUT:
                        time.sleep(0.0002)
                        continue
                    if rc != native.KATS_OK:
                        raise kats.KatsevichError(rc, msg)
                    out.popleft()
                    free.append(b)
                    lat[j] = (st["t_done_ms"] - st["t_submit_ms"]) + 1e3 * late
                    last_done = max(last_done, st["t_done_ms"])
                    if j == 0:
                        first_submit = st["t_submit_ms"] - 1e3 * late
                elif i < n_req:
                    time.sleep(max(0.0, min(0.001, arrivals[i] - now)))
            stats = srv.stats()
            stats["launches"] = native.katsevich_launch_count() - n_launch0
        return lat, (last_done - first_submit) / 1e3, stats

    clocks = Clocks(0)
    clocks.start()
    lat_sat, span_sat, st_sat = serve(None, True)
    runs = {}
    for rho in rhos:
        gaps = np.random.default_rng(seed).exponential(1.0 / (rho * mu), size=n_req)
        lat, span, st = serve(np.cumsum(gaps) - gaps[0], False)
        runs[str(rho)] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "vol_per_s": n_req / span, "max_running": st["max_running"]}
    clk = clocks.stop()
    upd = float(sum(updates[int(k)] for k in which))
    line = {
        "metric": METRIC, "value": n_req / span_sat, "unit": "vol/s", "n_gpus": 1, "steps": n_req, "warmup": len(protos),
        "ms_per_step": 1e3 * span_sat / n_req, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[args.precision], "data": "synthetic",
        "config": {"workload": "serving_mix_poisson_256", "protocols": len(protos), "requests": n_req,
                   "slots": slots, "arena_gb": args.arena_gb, "precision": args.precision,
                   "volumes": SERVING_VOLUMES, "views_per_turn": SERVING_VPT, "detector_cols": SERVING_DETECTORS,
                   "pitch_factors": SERVING_PITCH, "seed": seed},
        "serving": {
            "saturated": {"vol_per_s": n_req / span_sat, "gups": upd / span_sat / 1e9,
                          "p50_ms": float(np.percentile(lat_sat, 50)), "p99_ms": float(np.percentile(lat_sat, 99)),
                          "max_running": st_sat["max_running"], "arena_peak_gb": st_sat["arena_peak_bytes"] / 2**30},
            "poisson": runs,
            "plain_fp32": {"vol_per_s": mu, "gups": upd / plain_s / 1e9,
                           "note": "one request at a time through katsevich_recon_host (H2D, recon, D2H)"},
            "served_over_plain": (n_req / span_sat) / mu,
        },
        "gpu_launches": st_sat["launches"], "clocks": clk,
    }
    return line


# ----------------------------------------------------------- differentiation
def run_differentiation(args):
    print(json.dumps(differentiation_result(args)))


def differentiation_result(args):
    """Config 3: the operator as a differentiable layer.  One step = forward
    (steps 1-7) and backward (the hand-written adjoint) of a batch of 4
    sinograms of the sparse-detector scanner (368 columns, 580 views/turn,
    1.5 x max-fit pitch, 256 x 256 x 64 volume) through torch.autograd."""
    import torch

    import paper_2201_02309_b300 as kats
    import synth
    from paper_2201_02309_b300 import build
    from paper_2201_02309_b300.autograd import KatsevichLayer
    build.build()
    cfg = synth.config(3)
    g = kats.make_geometry(cfg)
    layer = KatsevichLayer(g)
    B = int(cfg["batch"])
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev).manual_seed(3)
    sino = torch.randn((B,) + layer.plan.sino_shape, generator=gen, device=dev).requires_grad_(True)
    cot = torch.randn((B,) + layer.plan.vol_shape, generator=gen, device=dev)
    upd = float(layer.plan.info["update_count"]) * B
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        layer(sino).backward(cot)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    clocks = Clocks(0)
    clocks.start()
    n_launch0 = kats.native.katsevich_launch_count()
    for i in range(args.steps):
        sino.grad = None
        ev[3 * i].record(st)
        vol = layer(sino)
        ev[3 * i + 1].record(st)
        vol.backward(cot)
        ev[3 * i + 2].record(st)
    torch.cuda.synchronize()
    launches = kats.native.katsevich_launch_count() - n_launch0
    clk = clocks.stop()
    fwd = statistics.mean(ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(args.steps))
    bwd = statistics.mean(ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(args.steps))
    line = {"metric": METRIC, "value": upd / (fwd + bwd) * 1e-6, "unit": "GUPS (forward + backward updates/s)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fwd + bwd,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"], "batch": B, "volume_xyz": [g["nx"], g["ny"], g["nz"]],
                       "detector_rows_cols": [g["n_rows"], g["n_cols"]], "views_per_turn": g["views_per_turn"],
                       "pitch_mm": g["P"], "updates_per_volume": upd / B},
            "forward_ms": fwd, "backward_ms": bwd, "forward_gups": upd / fwd * 1e-6, "backward_gups": upd / bwd * 1e-6,
            "gpu_launches": launches, "clocks": clk}
    return line


# ----------------------------------------------------------- data simulation
def run_simulate(args):
    """The paper's data generation on the clinical geometry (config 2): helical
    projection of a 512 x 512 x 256 label volume (all 9280 views), sparse
    detector (every 4th column) upsampled back, Gaussian+Poisson noise
    (I0 = 1e5, var = 0.5).  One step = one input sinogram."""
    import torch

    import paper_2201_02309_b300 as kats
    import synth
    from paper_2201_02309_b300 import build
    build.build()
    cfg = config_for(argparse.Namespace(config=2, nz=args.nz, turns=args.turns))
    g = kats.make_geometry(cfg)
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev).manual_seed(2)
    vol = torch.rand((g["nz"], g["ny"], g["nx"]), generator=gen, device=dev)
    rays = g["n_views"] * g["n_rows"] * g["n_cols"]
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        kats.simulate_input(g, vol, keep=4, seed=1)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * args.steps)]
    clocks = Clocks(0)
    clocks.start()
    n_launch0 = kats.native.katsevich_launch_count()
    for i in range(args.steps):
        ev[4 * i].record(st)
        g_gt = kats.project(g, vol)
        ev[4 * i + 1].record(st)
        g_up = kats.sparse_upsample(g, g_gt, 4)
        ev[4 * i + 2].record(st)
        kats.add_noise(g_up, I0=1e5, var=0.5, seed=i)
        ev[4 * i + 3].record(st)
    torch.cuda.synchronize()
    launches = kats.native.katsevich_launch_count() - n_launch0
    clk = clocks.stop()
    t_proj = statistics.mean(ev[4 * i].elapsed_time(ev[4 * i + 1]) for i in range(args.steps))
    t_up = statistics.mean(ev[4 * i + 1].elapsed_time(ev[4 * i + 2]) for i in range(args.steps))
    t_noise = statistics.mean(ev[4 * i + 2].elapsed_time(ev[4 * i + 3]) for i in range(args.steps))
    total = t_proj + t_up + t_noise
    line = {"metric": "data simulation rays/s (projection + sparse upsampling + noise)", "value": rays / total * 1e3,
            "unit": "rays/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (noise decisions f64)",
            "data": "synthetic", "config": {"workload": "simulate_" + cfg["name"], "views": g["n_views"],
                                            "keep": 4, "I0": 1e5, "var": 0.5},
            "stages_ms": {"project": t_proj, "sparse_upsample": t_up, "noise": t_noise},
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.simulate:
        run_simulate(args)
    elif args.config == 5:
        run_serving(args)
    elif args.config == 3:
        run_differentiation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
