"""The allocation-free entry point, for callers that cannot allocate device
memory (another component owns the allocator, or the memory budget is already
committed).  It must give the same result as the ordinary entry point, on two
calls in a row that share its fixed scratch array, and reject arrays whose
scratch would not fit.  This file is collected last."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


def test_noalloc_matches_context_entry_point_twice():
    import torch
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    torch.cuda.set_device(0)
    ctx = bm.Context(0)
    rng = np.random.default_rng(71)
    x1 = synth.ecg_signal(20000, 250.0, rng)
    y1, sp1 = synth.poisson_observe(x1, 50.0, rng)
    j2 = synth.config1()
    j3 = synth.config2()
    x4 = synth.texture_edge_image((512, 512), rng)
    y4, sp4 = synth.poisson_observe(x4, 5.0, rng)
    cases = [(y1, dict(noise=("poisson", sp1), patch=(32,), step=(4,), search=(129,), group_size=(16, 32))),
             (j2.y, j2.cfg), (j3.y, j3.cfg),
             (y4, dict(noise=("poisson", sp4), patch=(8, 8), step=(3, 3), search=(39, 39), group_size=(16, 32)))]
    for y, cfg in cases:
        ref = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
        ctx.bmnd_denoise(_cuda(y), ref, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"])
        refn = ref.cpu().numpy()
        for call in range(2):
            out = torch.full(y.shape, float("nan"), dtype=torch.float32, device="cuda:0")
            bm.bmnd_denoise_noalloc(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                                    cfg["group_size"])
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            PT.assert_voxels(got, refn, 1.0, what="noalloc call %d" % call)
    ctx.close()


def test_noalloc_rejects_arrays_beyond_its_scratch():
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros(2048, 2048, device="cuda:0")
    out = torch.empty_like(y)
    with pytest.raises(bm.BmndError) as e:
        bm.bmnd_denoise_noalloc(y, out, ("gaussian", 0.1), (8, 8), (3, 3), (39, 39), (16, 32))
    assert e.value.status == bm.ENOMEM
    assert "scratch" in str(e.value)
