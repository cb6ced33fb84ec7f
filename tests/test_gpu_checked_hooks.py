"""Two paths a healthy run never takes, driven by the checked build's test hooks (each case in a
child process with libkatsevich_debug.so; nothing here faults, traps or hangs the GPU).

* The device-timeout path.  The staged backprojection's producer stops issuing view pairs after
  a few of them (it arms no further copy), and the bounded mbarrier waits give up after 2^12
  polls instead of 2^22.  The consumers' waits run out, every CTA records KATS_ETIMEOUT in the
  plan's device status and retires with no copy in flight.  The reconstruction returns, the
  status reads as a timeout, a served request reports KATS_ETIMEOUT, and once the hooks are off
  the next call on the same plan equals a clean run bit for bit.
* The general end-weight path for plans whose PI windows are not monotone in z.  With the plan
  treated as non-monotone every view takes that path instead of the ramp walk; the volume must
  be the same bit for bit, and match the oracle.
Both for the single-group kernel (config-1 case) and for the slice-group kernel (a volume of four
pitches, where slices one to three pitches apart share a thread).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from cases import c1_case, check32, fourpitch_case

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path[:0] = [sys.argv[2], sys.argv[3]]
import cases
import paper_2201_02309_b300 as kats
from paper_2201_02309_b300 import native
from paper_2201_02309_b300.serving import Server

out = sys.argv[1]
rep = {"checked": native.katsevich_debug_checks_enabled()}
_, g, sino = cases.c1_case()
kp = kats.Plan(g)
d = torch.from_numpy(sino).cuda()
clean = kp.recon(d).cpu().numpy()
rep["status_clean"] = native.katsevich_device_status(kp.handle)

# the timeout path
native.katsevich_debug_wait_limit(1 << 12)
native.katsevich_debug_stall_producer(3)
stalled = torch.full(kp.vol_shape, float("nan"), device="cuda")  # CTAs that give up store nothing
kp.recon(d, out=stalled)
stalled = stalled.cpu().numpy()
rep["stalled_nan"] = int(np.isnan(stalled).sum())
rep["status_stalled"] = native.katsevich_device_status(kp.handle)
rep["status_after_read"] = native.katsevich_device_status(kp.handle)
rep["stalled_equal_clean"] = bool(np.array_equal(stalled, clean))
with Server(arena_bytes=1 << 30, plan_cache_bytes=1 << 30, slots=2) as srv:
    hs = torch.from_numpy(sino).pin_memory()
    t = srv.submit(g, hs)
    try:
        srv.wait(t)
        rep["served"] = 0
    except kats.KatsevichError as e:
        rep["served"] = e.status
    native.katsevich_debug_stall_producer(-1)
    native.katsevich_debug_wait_limit(0)
    t = srv.submit(g, hs)
    vol, _ = srv.wait(t)
    rep["served_after"] = bool(np.array_equal(vol.numpy(), clean))
again = kp.recon(d).cpu().numpy()
rep["again_equal_clean"] = bool(np.array_equal(again, clean))
rep["status_again"] = native.katsevich_device_status(kp.handle)

# the general end-weight path
native.katsevich_debug_nonmonotone(1)
general = kp.recon(d).cpu().numpy()
native.katsevich_debug_nonmonotone(0)
rep["general_equal_ramp"] = bool(np.array_equal(general, clean))
np.save(f"{out}/general.npy", general)
np.save(f"{out}/clean.npy", clean)

# the same two paths in the slice-group kernel (four and three groups of slices one pitch apart)
_, g4, sino4 = cases.fourpitch_case()
kp4 = kats.Plan(g4)
d4 = torch.from_numpy(sino4).cuda()
clean4 = kp4.recon(d4).cpu().numpy()
native.katsevich_debug_wait_limit(1 << 12)
native.katsevich_debug_stall_producer(3)
stalled4 = torch.full(kp4.vol_shape, float("nan"), device="cuda")
kp4.recon(d4, out=stalled4)
native.katsevich_debug_stall_producer(-1)
native.katsevich_debug_wait_limit(0)
rep["groups_stalled_nan"] = int(torch.isnan(stalled4).sum().item())
rep["groups_status_stalled"] = native.katsevich_device_status(kp4.handle)
rep["groups_again_equal_clean"] = bool(np.array_equal(kp4.recon(d4).cpu().numpy(), clean4))
native.katsevich_debug_nonmonotone(1)
general4 = kp4.recon(d4).cpu().numpy()
native.katsevich_debug_nonmonotone(0)
rep["groups_general_equal_ramp"] = bool(np.array_equal(general4, clean4))
np.save(f"{out}/general4.npy", general4)
rep["flags"] = native.katsevich_debug_check_flags()
print("REPORT " + json.dumps(rep))
"""


def test_timeout_path_and_general_window_path(tmp_path):
    from paper_2201_02309_b300 import build as kbuild
    kbuild.build(debug=True)
    env = dict(os.environ, KATSEVICH_DEBUG_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", CHILD, str(tmp_path), ROOT, HERE], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads([x for x in r.stdout.splitlines() if x.startswith("REPORT ")][-1][len("REPORT "):])
    print(rep)
    import paper_2201_02309_b300 as kats
    assert rep["checked"] == 1
    assert rep["status_clean"] == 0
    assert rep["status_stalled"] == 1  # a bounded device wait gave up
    assert rep["status_after_read"] == 0  # reading the status clears it
    assert not rep["stalled_equal_clean"] and rep["stalled_nan"] > 0  # the stalled volume is incomplete
    assert rep["served"] == kats.native.KATS_ETIMEOUT
    assert rep["served_after"] and rep["again_equal_clean"] and rep["status_again"] == 0
    assert rep["general_equal_ramp"]
    assert rep["groups_status_stalled"] == 1 and rep["groups_stalled_nan"] > 0
    assert rep["groups_again_equal_clean"] and rep["groups_general_equal_ramp"]
    assert rep["flags"] == 0
    _, g, sino = c1_case()
    want = oracle.Plan(g).recon(sino.astype(np.float64))
    check32(np.load(tmp_path / "general.npy"), want, name="general end-weight path")
    _, g4, sino4 = fourpitch_case()
    want4 = oracle.Plan(g4).recon(sino4.astype(np.float64))
    check32(np.load(tmp_path / "general4.npy"), want4, name="general end-weight path, slice groups")
