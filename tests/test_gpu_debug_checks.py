"""The bounds-checked build (KATS_DEBUG_CHECKS), the stand-in for a memory checker.

The staged-window kernels assume that every voxel's detector column lies inside its CTA's staged
view window and that every tap row they read unclamped lies inside the staged rows. The checked
build verifies both at every access. Each case runs in a child process with the checked library
and in one with the plain library. No invariant may be violated. The two builds must give the same
reconstruction bit for bit, and the same adjoint to within the run-to-run variation of its
global-atomic drains.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path[:0] = [sys.argv[2], sys.argv[3]]
import cases, synth
import paper_2201_02309_b300 as kats
from paper_2201_02309_b300 import native

out = sys.argv[1]
P = {"fp32": kats.KATS_PREC_FP32, "fp16": kats.KATS_PREC_FP16, "bf16": kats.KATS_PREC_BF16}
report = {"checked": native.katsevich_debug_checks_enabled(), "flags": {}}


def run(name, g, sino, precs=("fp32",), host=False):
    kp = kats.Plan(g)
    for prec in precs:
        vol = kp.recon(torch.from_numpy(sino).cuda(), precision=P[prec]).cpu().numpy()
        np.save(f"{out}/{name}_{prec}.npy", vol)
        if host:
            hv = torch.empty(kp.vol_shape, dtype=torch.float32).pin_memory()
            kp.recon_host(torch.from_numpy(sino).pin_memory(), hv, precision=P[prec])
            np.save(f"{out}/{name}_{prec}_host.npy", hv.numpy())
    y = np.random.default_rng(4).normal(size=kp.vol_shape).astype(np.float32)
    np.save(f"{out}/{name}_adjoint.npy", kp.adjoint(torch.from_numpy(y).cuda()).cpu().numpy())
    report["flags"][name] = native.katsevich_debug_check_flags()
    assert native.katsevich_device_status(kp.handle) == 0


_, g, sino = cases.c1_case()
run("c1", g, sino, ("fp32", "fp16", "bf16"))
_, g, sino = cases.odd_case()
run("odd", g, sino)
_, g, sino = cases.odd_case(tall=True)
run("odd_tall", g, sino, ("fp32", "fp16"))
for mode in (0, 1):
    _, g, sino = cases.multipitch_case(mode)
    run(f"multipitch{mode}", g, sino)
_, g, sino = cases.fourpitch_case()
run("fourpitch", g, sino, ("fp32", "fp16", "bf16"))
_, g, sino = cases.finevoxel_case()
run("finevoxel", g, sino, ("fp32", "bf16"))
_, g, sino = cases.narrow_case()
run("narrow", g, sino)
_, g = cases.c3_small_case()
run("c3_small", g, np.random.default_rng(6).normal(size=(g["n_views"], g["n_rows"], g["n_cols"])).astype(np.float32))
cfg = dict(synth.config(2))
cfg.update(nx=64, ny=64, nz=48)
g = kats.make_geometry(cfg)
kp0 = kats.Plan(g)
run("c2_column", g, np.random.default_rng(7).standard_normal(kp0.sino_shape).astype(np.float32),
    ("fp32", "fp16"), host=True)
# the clinical volume: every slice in a four- or three-group item, each view staged as a row band
g = kats.make_geometry(synth.config(2))
kp0 = kats.Plan(g)
run("c2_full", g, np.random.default_rng(10).standard_normal(kp0.sino_shape).astype(np.float32), ("fp32", "bf16"))
del kp0
# the column check is live: a window 16 columns too narrow must trip it (taps stay clamped)
_, g, sino = cases.c1_case()
kp = kats.Plan(g)
native.katsevich_debug_narrow_window(16)
kp.recon(torch.from_numpy(sino).cuda())
kp.adjoint(torch.from_numpy(np.ones(kp.vol_shape, np.float32)).cuda())
report["narrowed"] = native.katsevich_debug_check_flags()
native.katsevich_debug_narrow_window(0)
print("REPORT " + json.dumps(report))
"""


def run_child(checked: bool, out: str) -> dict:
    env = dict(os.environ, KATSEVICH_DEBUG_CHECKS="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", CHILD, out, ROOT, HERE], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("REPORT ")][-1]
    return json.loads(line[len("REPORT "):])


def test_checked_build_invariants_and_identity(tmp_path):
    from paper_2201_02309_b300 import build as kbuild
    kbuild.build(debug=True)
    dc, dp = tmp_path / "checked", tmp_path / "plain"
    dc.mkdir()
    dp.mkdir()
    checked = run_child(True, str(dc))
    plain = run_child(False, str(dp))
    assert checked["checked"] == 1 and plain["checked"] == 0
    assert all(v == 0 for v in checked["flags"].values()), checked["flags"]
    assert checked["narrowed"] & 1 and checked["narrowed"] & 4  # backprojection and adjoint column checks
    assert plain["narrowed"] == 0
    names = sorted(os.listdir(dc))
    assert names == sorted(os.listdir(dp)) and len(names) >= 26
    for n in names:
        a, b = np.load(dc / n), np.load(dp / n)
        if "adjoint" in n:  # window drains add with global float atomics: order varies run to run
            assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b), n
        else:
            assert np.array_equal(a, b), n
