"""katsevich_recon_noalloc: the full operator with the library's fixed device
scratch array instead of a caller workspace, for callers that cannot allocate
device memory at reconstruction time (memory reserved up front by another
allocator, or loops where an allocation's implicit synchronisation would stall
other streams).  Checked through the C ABI against katsevich_recon, bit for bit,
on two calls in a row with different inputs and on a batch of two, with every
library allocation made to fail during the call, and for its size limit.

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test when it gets here; it also runs alone.
"""
import numpy as np
import pytest

import oracle
import synth
from cases import c1_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2201_02309_b300 import build
    build.build()
    import paper_2201_02309_b300 as kats
    return torch, kats


def test_noalloc_matches_workspace_entry_point_twice(env):
    torch, kats = env
    _, g, sino = c1_case()
    plan = kats.Plan(g)
    nat = kats.native
    stream = torch.cuda.current_stream().cuda_stream
    # second call: different data, same shapes; third: a batch of two through the same array
    inputs = [sino[None], (0.5 * sino[::-1])[None], np.stack([sino, -2.0 * sino + 0.25])]
    for x in inputs:
        b = x.shape[0]
        d_sino = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        want = torch.empty((b,) + plan.vol_shape, dtype=torch.float32, device="cuda")
        got = torch.full((b,) + plan.vol_shape, float("nan"), dtype=torch.float32, device="cuda")
        ws = plan.workspace()
        nat.katsevich_recon(plan.handle, d_sino.data_ptr(), want.data_ptr(), b, nat.KATS_PREC_FP32,
                            ws.data_ptr(), ws.numel(), stream)
        torch.cuda.synchronize()
        # any device allocation by the library during the call would now fail with KATS_ENOMEM
        nat.katsevich_debug_fail_allocs(1000)
        try:
            nat.katsevich_recon_noalloc(plan.handle, d_sino.data_ptr(), got.data_ptr(), b, stream)
            torch.cuda.synchronize()
        finally:
            nat.katsevich_debug_fail_allocs(0)
        # the same kernels on the same inputs with the same layout: the same bits
        assert torch.equal(got, want)
        assert np.isfinite(got.cpu().numpy()).all()


def test_noalloc_rejects_oversized_geometry(env):
    torch, kats = env
    g = oracle.derive_geometry(synth.config(3))  # needs a few hundred MB of scratch
    plan = kats.Plan(g)
    assert plan.info["workspace_bytes"] > (64 << 20)
    d_sino = torch.zeros(plan.sino_shape, dtype=torch.float32, device="cuda")
    vol = torch.zeros(plan.vol_shape, dtype=torch.float32, device="cuda")
    with pytest.raises(kats.KatsevichError) as e:
        kats.native.katsevich_recon_noalloc(plan.handle, d_sino.data_ptr(), vol.data_ptr(), 1,
                                            torch.cuda.current_stream().cuda_stream)
    assert e.value.status == kats.native.KATS_ESPACE
    assert "static array holds" in str(e.value)
